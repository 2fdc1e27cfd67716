"""FP64 CPU oracle of the 3D central-moment lattice Boltzmann method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1202_6081_gb300``)
and neither imports the other.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, optional OpenMP over
cells); this module builds it with gcc, loads it with ctypes and wraps it for
numpy arrays.  State arrays use the paper's velocity order and the layout
``f[alpha][z][y][x]`` (x fastest), the same layout the CUDA path's
``lbm_get_state`` / ``lbm_set_state`` exchange.

Each function cites the passage of Premnath & Banerjee it follows:
  * ``lattice``           Sec. 2 (D3Q27 basis), App. A; App. G (D3Q15)
  * ``collide``           Sec. 4-8: source (App. C-E), cascade (Sec. 7)
  * ``source``            App. C-E (D3Q27), App. G (D3Q15)
  * ``run``               Eqs. cascadedcollision1 and cascadedstreaming1
  * ``macroscopic``       Eqs. densitycalculation, velocitycalculation
  * ``equilibrium``       not in the paper: attractor state minus S/2
  * ``collide_jacobian``  complex-step derivative of ``collide``
  * ``adjoint_step``      transpose of one ``run`` step (not in the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_INC = os.path.join(_HERE, "oracle_collide.inc")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

WALL_Y = 1
WALL_Z = 2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (-O2, OpenMP, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_INC))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_lattice.argtypes = [ctypes.c_int, ip, dp, dp, dp]
            lib.oracle_collide.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp, dp, dp, dp,
                                           dp, ctypes.c_int]
            lib.oracle_source.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp]
            lib.oracle_collide_jacobian.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp, dp,
                                                    ctypes.c_int]
            lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_uint, dp, dp, dp, dp, ctypes.c_int, dp,
                                       ctypes.c_int]
            lib.oracle_macroscopic.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp, dp, dp]
            lib.oracle_equilibrium.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp, dp, dp]
            lib.oracle_adjoint_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_uint, dp, dp, dp, dp,
                                                dp, dp, dp, ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, name):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (name, rc))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def lattice(Q: int):
    """Velocity set e[Q,3], basis K[alpha,beta] = K_beta(e_alpha), D[beta],
    and P[beta,alpha] = P_beta(e_alpha) (the relaxed central-moment
    polynomials at u = 0).  Sec. 2 / App. A (D3Q27), App. G (D3Q15)."""
    lib = _load()
    e = np.zeros((Q, 3), dtype=np.int32)
    K = np.zeros((Q, Q))
    D = np.zeros(Q)
    P = np.zeros((Q, Q))
    _check(lib.oracle_lattice(Q, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(K), _dp(D),
                              _dp(P)), "lattice")
    return e.astype(np.int64), K, D, P


def collide(Q: int, f, F, omega, nthreads: int = 0, want_A: bool = False):
    """Collision of independent cells: f [n,Q], F [n,3] -> (post [n,Q],
    g [n,Q], S [n,Q][, A [n,Q,Q]]).  Sec. 4-8 (cascade of Sec. 7)."""
    lib = _load()
    f = _c64(f)
    F = _c64(F)
    n = f.shape[0]
    om = _c64(omega)
    out = np.zeros_like(f)
    g = np.zeros_like(f)
    S = np.zeros_like(f)
    A = np.zeros((n, Q, Q)) if want_A else None
    _check(lib.oracle_collide(Q, n, _dp(f), _dp(F), _dp(om), _dp(out), _dp(g), _dp(S), _dp(A),
                              nthreads), "collide")
    return (out, g, S, A) if want_A else (out, g, S)


def source(Q: int, u, F):
    """Source term S(F, u) [n,Q] for u, F [n,3] (App. C-E; App. G)."""
    lib = _load()
    u = _c64(u)
    F = _c64(F)
    S = np.zeros((u.shape[0], Q))
    _check(lib.oracle_source(Q, u.shape[0], _dp(u), _dp(F), _dp(S)), "source")
    return S


def collide_jacobian(Q: int, f, F, omega, nthreads: int = 0):
    """J [n,Q,Q+3]: derivative of the post-collision state with respect to
    (f_0..f_{Q-1}, F_x, F_y, F_z), by the complex step."""
    lib = _load()
    f = _c64(f)
    F = _c64(F)
    n = f.shape[0]
    J = np.zeros((n, Q, Q + 3))
    _check(lib.oracle_collide_jacobian(Q, n, _dp(f), _dp(F), _dp(_c64(omega)), _dp(J), nthreads),
           "collide_jacobian")
    return J


def _force_args(F, N):
    """(field [3,N] or None, uniform [3]) from a force of shape (3,) or (3,N)."""
    F = _c64(F)
    if F.ndim == 1:
        return None, F
    return F.reshape(3, N), np.zeros(3)


def run(Q: int, shape, f, F, omega, nsteps: int, bc: int = 0, nthreads: int = 0):
    """``nsteps`` collide-and-stream steps of the state f [Q, nz, ny, nx]
    (Eqs. cascadedcollision1, cascadedstreaming1; half-way bounce-back on the
    faces named by ``bc``).  F: uniform (3,) or per cell (3, nz, ny, nx)."""
    lib = _load()
    nz, ny, nx = shape
    N = nx * ny * nz
    f = _c64(f).reshape(Q, N)
    Ff, Fu = _force_args(F, N)
    out = np.zeros_like(f)
    _check(lib.oracle_run(Q, nx, ny, nz, bc, _dp(f), _dp(Ff), _dp(Fu), _dp(_c64(omega)),
                          nsteps, _dp(out), nthreads), "run")
    return out.reshape(Q, nz, ny, nx)


def macroscopic(Q: int, f, F):
    """rho [N...], u [3, N...] (Eqs. densitycalculation, velocitycalculation)."""
    lib = _load()
    shp = f.shape[1:]
    N = int(np.prod(shp))
    f = _c64(f).reshape(Q, N)
    Ff, Fu = _force_args(F, N)
    rho = np.zeros(N)
    u = np.zeros((3, N))
    _check(lib.oracle_macroscopic(Q, N, _dp(f), _dp(Ff), _dp(Fu), _dp(rho), _dp(u)),
           "macroscopic")
    return rho.reshape(shp), u.reshape((3,) + shp)


def equilibrium(Q: int, rho, u, F):
    """Initial state f = f^at(rho, u) - S/2 [Q, ...] for rho [...], u [3, ...]."""
    lib = _load()
    shp = np.shape(rho)
    N = int(np.prod(shp))
    r = _c64(rho).reshape(N)
    uu = _c64(u).reshape(3, N)
    Ff, Fu = _force_args(F, N)
    f = np.zeros((Q, N))
    _check(lib.oracle_equilibrium(Q, N, _dp(r), _dp(uu), _dp(Ff), _dp(Fu), _dp(f)),
           "equilibrium")
    return f.reshape((Q,) + shp)


def adjoint_step(Q: int, shape, f, F, omega, lam_next, bc: int = 0, gF=None,
                 nthreads: int = 0):
    """Transpose of one collide-and-stream step taken from state f: returns
    lam = (d f_next / d f)^T lam_next and, when gF [3, ...] is given, adds
    (d f_next / d F)^T lam_next to it in place."""
    lib = _load()
    nz, ny, nx = shape
    N = nx * ny * nz
    f = _c64(f).reshape(Q, N)
    ln = _c64(lam_next).reshape(Q, N)
    Ff, Fu = _force_args(F, N)
    lam = np.zeros((Q, N))
    gbuf = None
    if gF is not None:
        gbuf = _c64(gF).reshape(3, N).copy()
    _check(lib.oracle_adjoint_step(Q, nx, ny, nz, bc, _dp(f), _dp(Ff), _dp(Fu),
                                   _dp(_c64(omega)), _dp(ln), _dp(lam), _dp(gbuf), nthreads),
           "adjoint_step")
    if gF is not None:
        gF[...] = gbuf.reshape(gF.shape)
    return lam.reshape((Q, nz, ny, nx))


def kinetic_energy(Q: int, f, F):
    """J = sum_x rho |u|^2 / 2 with u from Eq. velocitycalculation."""
    rho, u = macroscopic(Q, f, F)
    return float(0.5 * np.sum(rho * np.sum(u * u, axis=0)))


def macroscopic_grad(Q: int, f, F, g_rho, g_u):
    """Chain rule through Eqs. densitycalculation and velocitycalculation:
    for J(rho, u) with dJ/drho = g_rho [...] and dJ/du = g_u [3, ...],
    dJ/df_alpha = g_rho + sum_i (e_alpha,i - u_i) g_u_i / rho (rho = sum f,
    rho u = sum f e + F/2) and the direct dJ/dF_i = g_u_i / (2 rho)."""
    e, _, _, _ = lattice(Q)
    rho, u = macroscopic(Q, f, F)
    g_rho = np.broadcast_to(np.asarray(g_rho, dtype=np.float64), rho.shape)
    g_u = np.asarray(g_u, dtype=np.float64)
    dfl = np.stack([g_rho + sum((e[a, i] - u[i]) * g_u[i] for i in range(3)) / rho
                    for a in range(Q)])
    return dfl, g_u / (2.0 * rho)


def kinetic_energy_grad(Q: int, f, F):
    """dJ/df [Q, ...] and the direct dJ/dF [3, ...] of ``kinetic_energy``:
    with j = sum f e + F/2, J = |j|^2 / (2 rho), so dJ/df_alpha =
    u.e_alpha - |u|^2 / 2 and dJ/dF_i = u_i / 2."""
    e, _, _, _ = lattice(Q)
    rho, u = macroscopic(Q, f, F)
    u2 = np.sum(u * u, axis=0)
    dfl = np.stack([e[a, 0] * u[0] + e[a, 1] * u[1] + e[a, 2] * u[2] - 0.5 * u2
                    for a in range(Q)])
    return dfl, 0.5 * u
