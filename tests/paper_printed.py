"""The paper's printed closed-form expressions, transcribed for the tests.

These are the formulas Premnath & Banerjee print for a faster evaluation of
the method: raw moments through index sets (App. B, App. G), raw source
moments (App. C), their projections m^s (App. D, App. G), the D3Q15 source
rows (App. G) and the explicit cascaded collision kernels g_4..g_26 (Sec. 7)
and g_4..g_14 (App. G).  The oracle computes the same quantities from their
definitions (basis polynomials, binomial theorem, exact inversion, cascade
rule), so agreement between the two pins the oracle.

Seven printed D3Q27 coefficients disagree with the definition; each is
marked "reading:" below with the corrected form used here.  The D3Q15
kernels are used exactly as printed.

Every function takes cell-major arrays: f [n,Q], F [n,3], omega [Q].
"""
import numpy as np

# App. B: index sets A_k (+1) and B_k (-1) of the D3Q27 raw moments.
IDX27 = {
    "xy": ([7, 10, 19, 22, 23, 26], [8, 9, 20, 21, 24, 25]),
    "xz": ([11, 14, 19, 21, 24, 26], [12, 13, 20, 22, 23, 25]),
    "yz": ([15, 18, 19, 20, 25, 26], [16, 17, 21, 22, 23, 24]),
    "xx": ([1, 2, 7, 8, 9, 10, 11, 12, 13, 14, 19, 20, 21, 22, 23, 24, 25, 26], []),
    "yy": ([3, 4, 7, 8, 9, 10, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26], []),
    "zz": ([5, 6, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26], []),
    "xyy": ([7, 9, 19, 21, 23, 25], [8, 10, 20, 22, 24, 26]),
    "xzz": ([11, 13, 19, 21, 23, 25], [12, 14, 20, 22, 24, 26]),
    "xxy": ([7, 8, 19, 20, 23, 24], [9, 10, 21, 22, 25, 26]),
    "yzz": ([15, 17, 19, 20, 23, 24], [16, 18, 21, 22, 25, 26]),
    "xxz": ([11, 12, 19, 20, 21, 22], [13, 14, 23, 24, 25, 26]),
    "yyz": ([15, 16, 19, 20, 21, 22], [17, 18, 23, 24, 25, 26]),
    "xyz": ([19, 22, 24, 25], [20, 21, 23, 26]),
    "xxyy": ([7, 8, 9, 10, 19, 20, 21, 22, 23, 24, 25, 26], []),
    "xxzz": ([11, 12, 13, 14, 19, 20, 21, 22, 23, 24, 25, 26], []),
    "yyzz": ([15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26], []),
    "xxyz": ([19, 20, 25, 26], [21, 22, 23, 24]),
    "xyyz": ([19, 21, 24, 26], [20, 22, 23, 25]),
    "xyzz": ([19, 22, 23, 26], [20, 21, 24, 25]),
    "xyyzz": ([19, 21, 23, 25], [20, 22, 24, 26]),
    "xxyzz": ([19, 20, 23, 24], [21, 22, 25, 26]),
    "xxyyz": ([19, 20, 21, 22], [23, 24, 25, 26]),
    "xxyyzz": ([19, 20, 21, 22, 23, 24, 25, 26], []),
}

# App. G: index sets of the D3Q15 raw moments.
IDX15 = {
    "xy": ([7, 10, 11, 14], [8, 9, 12, 13]),
    "xz": ([7, 9, 12, 14], [8, 10, 11, 13]),
    "yz": ([7, 8, 13, 14], [9, 10, 11, 12]),
    "xx": ([1, 2, 7, 8, 9, 10, 11, 12, 13, 14], []),
    "yy": ([3, 4, 7, 8, 9, 10, 11, 12, 13, 14], []),
    "zz": ([5, 6, 7, 8, 9, 10, 11, 12, 13, 14], []),
    "xyy": ([7, 9, 11, 13], [8, 10, 12, 14]),
    "xxy": ([7, 8, 11, 12], [9, 10, 13, 14]),
    "xxz": ([7, 8, 9, 10], [11, 12, 13, 14]),
    "xyz": ([7, 10, 12, 13], [8, 9, 11, 14]),
    "xxyy": ([7, 8, 9, 10, 11, 12, 13, 14], []),
}


def raw_moments(f, idx):
    """kappa-bar' from the index sets: sum over A minus sum over B."""
    return {k: f[:, a].sum(axis=1) - (f[:, b].sum(axis=1) if b else 0.0)
            for k, (a, b) in idx.items()}


def raw_source_moments(F, u):
    """App. C: raw source moments sigma' of the de-aliased forcing."""
    Fx, Fy, Fz = F[:, 0], F[:, 1], F[:, 2]
    ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
    return {
        "x": Fx, "y": Fy, "z": Fz,
        "xx": 2 * Fx * ux, "yy": 2 * Fy * uy, "zz": 2 * Fz * uz,
        "xy": Fx * uy + Fy * ux, "xz": Fx * uz + Fz * ux, "yz": Fy * uz + Fz * uy,
        "xyy": Fx * uy**2 + 2 * Fy * uy * ux, "xzz": Fx * uz**2 + 2 * Fz * uz * ux,
        "xxy": Fy * ux**2 + 2 * Fx * ux * uy, "yzz": Fy * uz**2 + 2 * Fz * uz * uy,
        "xxz": Fz * ux**2 + 2 * Fx * ux * uz, "yyz": Fz * uy**2 + 2 * Fy * uy * uz,
        "xyz": Fx * uy * uz + Fy * ux * uz + Fz * ux * uy,
        "xxyy": 2 * Fx * ux * uy**2 + 2 * Fy * uy * ux**2,
        "xxzz": 2 * Fx * ux * uz**2 + 2 * Fz * uz * ux**2,
        "yyzz": 2 * Fy * uy * uz**2 + 2 * Fz * uz * uy**2,
        "xxyz": ux**2 * (Fy * uz + Fz * uy) + 2 * Fx * ux * uy * uz,
        "xyyz": uy**2 * (Fx * uz + Fz * ux) + 2 * Fy * uy * ux * uz,
        "xyzz": uz**2 * (Fx * uy + Fy * ux) + 2 * Fz * uz * ux * uy,
        "xyyzz": Fx * uy**2 * uz**2 + 2 * ux * uy * uz * (Fy * uz + Fz * uy),
        "xxyzz": Fy * ux**2 * uz**2 + 2 * ux * uy * uz * (Fx * uz + Fz * ux),
        "xxyyz": Fz * ux**2 * uy**2 + 2 * ux * uy * uz * (Fx * uy + Fy * ux),
        "xxyyzz": 2 * ux * uy * uz * (Fx * uy * uz + Fy * uz * ux + Fz * ux * uy),
    }


def ms_q27(F, u):
    """App. D: projections m^s_beta = <K_beta|S> on D3Q27."""
    Fx, Fy, Fz = F[:, 0], F[:, 1], F[:, 2]
    ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
    m = np.zeros((F.shape[0], 27))
    m[:, 1], m[:, 2], m[:, 3] = Fx, Fy, Fz
    m[:, 4] = Fx * uy + Fy * ux
    m[:, 5] = Fx * uz + Fz * ux
    m[:, 6] = Fy * uz + Fz * uy
    m[:, 7] = 2 * (Fx * ux - Fy * uy)
    m[:, 8] = 2 * (Fx * ux + Fy * uy - 2 * Fz * uz)
    m[:, 9] = 2 * (Fx * ux + Fy * uy + Fz * uz)
    m[:, 10] = 3 * (Fx * (uy**2 + uz**2) + 2 * ux * (Fy * uy + Fz * uz)) - 4 * Fx
    m[:, 11] = 3 * (Fy * (ux**2 + uz**2) + 2 * uy * (Fx * ux + Fz * uz)) - 4 * Fy
    m[:, 12] = 3 * (Fz * (ux**2 + uy**2) + 2 * uz * (Fx * ux + Fy * uy)) - 4 * Fz
    m[:, 13] = Fx * (uy**2 - uz**2) + 2 * ux * (Fy * uy - Fz * uz)
    m[:, 14] = Fy * (ux**2 - uz**2) + 2 * uy * (Fx * ux - Fz * uz)
    m[:, 15] = Fz * (ux**2 - uy**2) + 2 * uz * (Fx * ux - Fy * uy)
    m[:, 16] = Fx * uy * uz + Fy * ux * uz + Fz * ux * uy
    m[:, 17] = (6 * (Fx * ux * (uy**2 + uz**2) + Fy * uy * (ux**2 + uz**2)
                     + Fz * uz * (ux**2 + uy**2)) - 8 * (Fx * ux + Fy * uy + Fz * uz))
    m[:, 18] = (6 * (Fx * ux * (uy**2 + uz**2) + Fy * uy * (ux**2 - 2 * uz**2)
                     + Fz * uz * (ux**2 - 2 * uy**2)) - 4 * (2 * Fx * ux - Fy * uy - Fz * uz))
    m[:, 19] = 6 * (Fx * ux * (uy**2 - uz**2) + ux**2 * (Fy * uy - Fz * uz)) - 4 * (Fy * uy - Fz * uz)
    m[:, 20] = (3 * ux**2 - 2) * (Fy * uz + Fz * uy) + 6 * Fx * ux * uy * uz
    m[:, 21] = (3 * uy**2 - 2) * (Fx * uz + Fz * ux) + 6 * Fy * uy * ux * uz
    m[:, 22] = (3 * uz**2 - 2) * (Fx * uy + Fy * ux) + 6 * Fz * uz * ux * uy
    m[:, 23] = (9 * Fx * (uy**2 * uz**2 - 2.0 / 3.0 * ((uy**2 + uz**2) - 2.0 / 3.0))
                + 18 * ux * (Fy * uy * uz**2 + Fz * uz * uy**2 - 2.0 / 3.0 * (Fy * uy + Fz * uz)))
    m[:, 24] = (9 * Fy * (ux**2 * uz**2 - 2.0 / 3.0 * ((ux**2 + uz**2) - 2.0 / 3.0))
                + 18 * uy * (Fx * ux * uz**2 + Fz * uz * ux**2 - 2.0 / 3.0 * (Fx * ux + Fz * uz)))
    m[:, 25] = (9 * Fz * (ux**2 * uy**2 - 2.0 / 3.0 * ((ux**2 + uy**2) - 2.0 / 3.0))
                + 18 * uz * (Fx * ux * uy**2 + Fy * uy * ux**2 - 2.0 / 3.0 * (Fx * ux + Fy * uy)))
    m[:, 26] = (Fx * ux * (54 * uy**2 * uz**2 - 36 * (uy**2 + uz**2) + 24)
                + Fy * uy * (54 * ux**2 * uz**2 - 36 * (ux**2 + uz**2) + 24)
                + Fz * uz * (54 * ux**2 * uy**2 - 36 * (ux**2 + uy**2) + 24))
    return m


def ms_q15(F, u):
    """App. G: projections m^s_beta = <K_beta|S> on D3Q15."""
    Fx, Fy, Fz = F[:, 0], F[:, 1], F[:, 2]
    ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
    m = np.zeros((F.shape[0], 15))
    m[:, 1], m[:, 2], m[:, 3] = Fx, Fy, Fz
    m[:, 4] = Fx * uy + Fy * ux
    m[:, 5] = Fx * uz + Fz * ux
    m[:, 6] = Fy * uz + Fz * uy
    m[:, 7] = 2 * (Fx * ux - Fy * uy)
    m[:, 8] = 2 * (Fx * ux + Fy * uy - 2 * Fz * uz)
    m[:, 9] = 2 * (Fx * ux + Fy * uy + Fz * uz)
    m[:, 10] = 5 * (Fx * (3 * ux**2 + uy**2 + uz**2) + 2 * ux * (Fy * uy + Fz * uz)) - 13 * Fx
    m[:, 11] = 5 * (Fy * (ux**2 + 3 * uy**2 + uz**2) + 2 * uy * (Fx * ux + Fz * uz)) - 13 * Fy
    m[:, 12] = 5 * (Fz * (ux**2 + uy**2 + 3 * uz**2) + 2 * uz * (Fx * ux + Fy * uy)) - 13 * Fz
    m[:, 13] = Fx * uy * uz + Fy * ux * uz + Fz * ux * uy
    m[:, 14] = 20 * (Fx * ux * (3 * (uy**2 + uz**2) - 4) + Fy * uy * (3 * (ux**2 + uz**2) - 4)
                     + Fz * uz * (3 * (ux**2 + uy**2) - 4))
    return m


def source_q15(m):
    """App. G: the D3Q15 source rows S_alpha in terms of m^s."""
    S = np.zeros_like(m)
    S[:, 0] = (3 * m[:, 0] - 5 * m[:, 9] + m[:, 14]) / 45
    S[:, 1] = (12 * m[:, 0] + 18 * m[:, 1] + 45 * m[:, 7] + 15 * m[:, 8] - 10 * m[:, 9]
               - 9 * m[:, 10] - m[:, 14]) / 180
    S[:, 2] = (12 * m[:, 0] - 18 * m[:, 1] + 45 * m[:, 7] + 15 * m[:, 8] - 10 * m[:, 9]
               + 9 * m[:, 10] - m[:, 14]) / 180
    S[:, 3] = (12 * m[:, 0] + 18 * m[:, 2] - 45 * m[:, 7] + 15 * m[:, 8] - 10 * m[:, 9]
               - 9 * m[:, 11] - m[:, 14]) / 180
    S[:, 4] = (12 * m[:, 0] - 18 * m[:, 2] - 45 * m[:, 7] + 15 * m[:, 8] - 10 * m[:, 9]
               + 9 * m[:, 11] - m[:, 14]) / 180
    S[:, 5] = (12 * m[:, 0] + 18 * m[:, 3] - 30 * m[:, 8] - 10 * m[:, 9] - 9 * m[:, 12]
               - m[:, 14]) / 180
    S[:, 6] = (12 * m[:, 0] - 18 * m[:, 3] - 30 * m[:, 8] - 10 * m[:, 9] + 9 * m[:, 12]
               - m[:, 14]) / 180
    # S_7..S_14: 48 m0 + 72 (sx m1 + sy m2 + sz m3) + 90 (sxsy m4 + sxsz m5 + sysz m6)
    #            + 40 m9 + 9 (sx m10 + sy m11 + sz m12) + 90 sxsysz m13 + m14, over 720
    corners = [(1, 1, 1), (-1, 1, 1), (1, -1, 1), (-1, -1, 1),
               (1, 1, -1), (-1, 1, -1), (1, -1, -1), (-1, -1, -1)]
    for k, (sx, sy, sz) in enumerate(corners):
        S[:, 7 + k] = (48 * m[:, 0] + 72 * (sx * m[:, 1] + sy * m[:, 2] + sz * m[:, 3])
                       + 90 * (sx * sy * m[:, 4] + sx * sz * m[:, 5] + sy * sz * m[:, 6])
                       + 40 * m[:, 9] + 9 * (sx * m[:, 10] + sy * m[:, 11] + sz * m[:, 12])
                       + 90 * sx * sy * sz * m[:, 13] + m[:, 14]) / 720
    return S


def _macro(f, F, e):
    rho = f.sum(axis=1)
    u = (f @ e + 0.5 * F) / rho[:, None]
    return rho, u


def kernels_q27(f, F, om, e):
    """Sec. 7: printed D3Q27 collision kernels g_4..g_26, with seven readings.
    Returns (g [n,27], (kxx, kyy, kzz))."""
    rho, u = _macro(f, F, e)
    ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
    kb = raw_moments(f, IDX27)
    sg = raw_source_moments(F, u)
    E = {k: kb[k] + sg[k] for k in kb}  # eta' = kappa-bar' + sigma'
    sx, sy, sz = sg["x"], sg["y"], sg["z"]
    exy, exz, eyz = E["xy"], E["xz"], E["yz"]
    exx, eyy, ezz = E["xx"], E["yy"], E["zz"]
    exyy, exzz, exxy, eyzz, exxz, eyyz, exyz = (E["xyy"], E["xzz"], E["xxy"], E["yzz"], E["xxz"],
                                                E["yyz"], E["xyz"])
    exxyy, exxzz, eyyzz = E["xxyy"], E["xxzz"], E["yyzz"]
    exxyz, exyyz, exyzz = E["xxyz"], E["xyyz"], E["xyzz"]
    exyyzz, exxyzz, exxyyz, exxyyzz = E["xyyzz"], E["xxyzz"], E["xxyyz"], E["xxyyzz"]
    w = om
    g4 = w[4] / 12 * (-exy + rho * ux * uy + 0.5 * (sx * uy + sy * ux))
    g5 = w[5] / 12 * (-exz + rho * ux * uz + 0.5 * (sx * uz + sz * ux))
    g6 = w[6] / 12 * (-eyz + rho * uy * uz + 0.5 * (sy * uz + sz * uy))
    g7 = w[7] / 12 * (-(exx - eyy) + rho * (ux**2 - uy**2) + (sx * ux - sy * uy))
    g8 = w[8] / 36 * (-(exx + eyy - 2 * ezz) + rho * (ux**2 + uy**2 - 2 * uz**2)
                      + (sx * ux + sy * uy - 2 * sz * uz))
    g9 = w[9] / 18 * (-(exx + eyy + ezz) + rho * (ux**2 + uy**2 + uz**2)
                      + (sx * ux + sy * uy + sz * uz) + rho)
    g10 = (w[10] / 24 * (-(exyy + exzz) + 2 * (uy * exy + uz * exz) + ux * (eyy + ezz)
                         - 2 * rho * ux * (uy**2 + uz**2) - 0.5 * sx * (uy**2 + uz**2)
                         - ux * (sy * uy + sz * uz))
           + (uy * g4 + uz * g5) + 0.25 * ux * (-g7 - g8 + 2 * g9))
    g11 = (w[11] / 24 * (-(exxy + eyzz) + 2 * (ux * exy + uz * eyz) + uy * (exx + ezz)
                         - 2 * rho * uy * (ux**2 + uz**2) - 0.5 * sy * (ux**2 + uz**2)
                         - uy * (sx * ux + sz * uz))
           + (ux * g4 + uz * g6) + 0.25 * uy * (g7 - g8 + 2 * g9))
    g12 = (w[12] / 24 * (-(exxz + eyyz) + 2 * (ux * exz + uy * eyz) + uz * (exx + eyy)
                         - 2 * rho * uz * (ux**2 + uy**2) - 0.5 * sz * (ux**2 + uy**2)
                         - uz * (sx * ux + sy * uy))
           + (ux * g5 + uy * g6) + 0.5 * uz * (g8 + g9))
    g13 = (w[13] / 8 * (-(exyy - exzz) + 2 * (uy * exy - uz * exz) + ux * (eyy - ezz)
                        - 2 * rho * ux * (uy**2 - uz**2) - 0.5 * sx * (uy**2 - uz**2)
                        - ux * (sy * uy - sz * uz))
           + 3 * (uy * g4 - uz * g5) + 0.75 * ux * (-g7 + 3 * g8))
    g14 = (w[14] / 8 * (-(exxy - eyzz) + 2 * (ux * exy - uz * eyz) + uy * (exx - ezz)
                        - 2 * rho * uy * (ux**2 - uz**2) - 0.5 * sy * (ux**2 - uz**2)
                        - uy * (sx * ux - sz * uz))
           + 3 * (ux * g4 - uz * g6) + 0.75 * uy * (g7 + 3 * g8))
    g15 = (w[15] / 8 * (-(exxz - eyyz) + 2 * (ux * exz - uy * eyz) + uz * (exx - eyy)
                        - 2 * rho * uz * (ux**2 - uy**2) - 0.5 * sz * (ux**2 - uy**2)
                        - uz * (sx * ux - sy * uy))
           + 3 * (ux * g5 - uy * g6) + 1.5 * uz * g7)
    # reading: the last term of g_16 is printed u_z g_6; the definition gives u_x g_6.
    g16 = (w[16] / 8 * (-exyz + ux * eyz + uy * exz + uz * exy - 2 * rho * ux * uy * uz
                        - 0.5 * (sx * uy * uz + sy * ux * uz + sz * ux * uy))
           + 1.5 * (uz * g4 + uy * g5 + ux * g6))
    kxx = (exx + 6 * g7 + 6 * g8 + 6 * g9) - rho * ux**2 - F[:, 0] * ux
    kyy = (eyy - 6 * g7 + 6 * g8 + 6 * g9) - rho * uy**2 - F[:, 1] * uy
    # reading: kappa~_zz is printed with eta'_xx; the definition gives eta'_zz.
    kzz = (ezz - 12 * g8 + 6 * g9) - rho * uz**2 - F[:, 2] * uz
    # reading: the g_9 coefficient of g_17 is printed (-2ux^2-2uy^2-uz^2-4)/2;
    # the definition gives (-2ux^2-2uy^2-2uz^2-4)/2.
    g17 = (w[17] / 12 * (-(exxyy + exxzz + eyyzz)
                         + 2 * (ux * (exyy + exzz) + uy * (eyzz + exxy) + uz * (exxz + eyyz))
                         - ux**2 * (eyy + ezz) - uy**2 * (exx + ezz) - uz**2 * (exx + eyy)
                         - 4 * (ux * uy * exy + ux * uz * exz + uy * uz * eyz)
                         + (kxx * kyy + kxx * kzz + kyy * kzz)
                         + 3 * rho * (ux**2 * uy**2 + ux**2 * uz**2 + uy**2 * uz**2)
                         + ux**2 * (uy * sy + uz * sz) + uy**2 * (ux * sx + uz * sz)
                         + uz**2 * (ux * sx + uy * sy))
           - 4 * ux * uy * g4 - 4 * ux * uz * g5 - 4 * uy * uz * g6
           + 0.5 * (ux**2 - uy**2) * g7 + 0.5 * (ux**2 + uy**2 - 2 * uz**2) * g8
           + 0.5 * (-2 * ux**2 - 2 * uy**2 - 2 * uz**2 - 4) * g9
           + 4 * ux * g10 + 4 * uy * g11 + 4 * uz * g12)
    # reading: the g_9 coefficient of g_18 is printed (-2ux^2+uy^2+2uz^2)/4;
    # the definition gives (-2ux^2+uy^2+uz^2)/4.
    g18 = (w[18] / 24 * (-(exxyy + exxzz - 2 * eyyzz)
                         + 2 * (ux * exyy + ux * exzz + uy * exxy + uz * exxz
                                - 2 * (uy * eyzz + uz * eyyz))
                         - ux**2 * eyy - ux**2 * ezz - uy**2 * exx - uz**2 * exx
                         + 2 * uy**2 * ezz + 2 * uz**2 * eyy
                         - 4 * (ux * uy * exy + ux * uz * exz - 2 * uy * uz * eyz)
                         + (kxx * kyy + kxx * kzz - 2 * kyy * kzz)
                         + 3 * rho * (ux**2 * uy**2 + ux**2 * uz**2 - 2 * uy**2 * uz**2)
                         + ux**2 * uy * sy + ux**2 * uz * sz + uy**2 * ux * sx + uz**2 * ux * sx
                         - 2 * uy**2 * uz * sz - 2 * uz**2 * uy * sy)
           - 2 * ux * uy * g4 - 2 * ux * uz * g5 + 4 * uy * uz * g6
           + 0.25 * (ux**2 - uy**2 - 3 * uz**2 - 2) * g7
           + 0.25 * (ux**2 - 5 * uy**2 + uz**2 - 2) * g8
           + 0.25 * (-2 * ux**2 + uy**2 + uz**2) * g9
           + 2 * ux * g10 - uy * g11 - uz * g12 + uy * g14 + uz * g15)
    # reading: the g_9 coefficient of g_19 is printed (-3uy^2-8)/4; the
    # definition gives (-3uy^2+3uz^2)/4.
    g19 = (w[19] / 8 * (-(exxyy - exxzz)
                        + 2 * (ux * exyy - ux * exzz + uy * exxy - uz * exxz)
                        - (ux**2 * eyy - ux**2 * ezz + uy**2 * exx - uz**2 * exx)
                        - 4 * (ux * uy * exy - ux * uz * exz)
                        + (kxx * kyy - kxx * kzz) + 3 * rho * (ux**2 * uy**2 - ux**2 * uz**2)
                        + (ux**2 * uy * sy - ux**2 * uz * sz + uy**2 * ux * sx - uz**2 * ux * sx))
           - 6 * ux * uy * g4 + 6 * ux * uz * g5
           + 0.25 * (3 * ux**2 - 3 * uy**2 + 3 * uz**2 + 2) * g7
           + 0.25 * (-9 * ux**2 - 3 * uy**2 + 3 * uz**2 - 6) * g8
           + 0.25 * (-3 * uy**2 + 3 * uz**2) * g9
           + 3 * uy * g11 - 3 * uz * g12 + 2 * ux * g13 + uy * g14 - uz * g15)
    g20 = (w[20] / 8 * (-exxyz + uz * exxy + uy * exxz + 2 * ux * exyz - uy * uz * exx
                        - 2 * ux * uz * exy - 2 * ux * uy * exz - ux**2 * eyz
                        + 3 * rho * ux**2 * uy * uz + sx * ux * uy * uz
                        + 0.5 * ux**2 * (sy * uz + sz * uy))
           - 3 * ux * uz * g4 - 3 * ux * uy * g5 - (1.5 * ux**2 + 1) * g6
           - 0.75 * uy * uz * g7 - 0.75 * uy * uz * g8 - 0.75 * uy * uz * g9
           + 1.5 * uz * g11 + 1.5 * uy * g12 + 0.5 * uz * g14 + 0.5 * uy * g15 + 2 * ux * g16)
    g21 = (w[21] / 8 * (-exyyz + 2 * uy * exyz + uz * exyy + ux * eyyz - uy**2 * exz
                        - 2 * uy * uz * exy - 2 * ux * uy * eyz - ux * uz * eyy
                        + 3 * rho * ux * uy**2 * uz + sy * ux * uy * uz
                        + 0.5 * uy**2 * (sx * uz + sz * ux))
           - 3 * uy * uz * g4 - (1.5 * uy**2 + 1) * g5 - 3 * ux * uy * g6
           + 0.75 * ux * uz * g7 - 0.75 * ux * uz * g8 - 0.75 * ux * uz * g9
           + 1.5 * uz * g10 + 1.5 * ux * g12 + 0.5 * uz * g13 - 0.5 * ux * g15 + 2 * uy * g16)
    g22 = (w[22] / 8 * (-exyzz + 2 * uz * exyz + uy * exzz + ux * eyzz - uz**2 * exy
                        - 2 * uy * uz * exz - 2 * ux * uz * eyz - ux * uy * ezz
                        + 3 * rho * ux * uy * uz**2 + sz * ux * uy * uz
                        + 0.5 * uz**2 * (sx * uy + sy * ux))
           - (1.5 * uz**2 + 1) * g4 - 3 * uy * uz * g5 - 3 * ux * uz * g6
           + 1.5 * ux * uy * g8 - 0.75 * ux * uy * g9
           + 1.5 * uy * g10 + 1.5 * ux * g11 - 0.5 * uy * g13 - 0.5 * ux * g14 + 2 * uz * g16)
    # reading: the g_7 coefficient of g_23 is printed (3/4 ux uz^2 - 1/4 ux);
    # the definition gives (-3/4 ux uz^2 - 1/2 ux).
    g23 = (w[23] / 8 * (-exyyzz + ux * eyyzz + 2 * uy * exyzz + 2 * uz * exyyz - uy**2 * exzz
                        - uz**2 * exyy - 2 * ux * uy * eyzz - 2 * ux * uz * eyyz
                        - 4 * uy * uz * exyz + ux * uz**2 * eyy + ux * uy**2 * ezz
                        + 2 * uy * uz**2 * exy + 2 * uy**2 * uz * exz + 4 * ux * uy * uz * eyz
                        - 4 * rho * ux * uy**2 * uz**2 - 0.5 * uy**2 * uz**2 * sx
                        - ux * (uz**2 * uy * sy + uy**2 * uz * sz))
           + (3 * uy * uz**2 + 2 * uy) * g4 + (3 * uy**2 * uz + 2 * uz) * g5
           + 6 * ux * uy * uz * g6 + (-0.75 * ux * uz**2 - 0.5 * ux) * g7
           + (0.75 * ux * uz**2 - 1.5 * ux * uy**2 - 0.5 * ux) * g8
           + (0.75 * ux * uz**2 + 0.75 * ux * uy**2 + ux) * g9
           + (-1.5 * uy**2 - 1.5 * uz**2 - 2) * g10 - 3 * ux * uy * g11
           - 3 * ux * uz * g12 + (0.5 * uy**2 - 0.5 * uz**2) * g13 + ux * uy * g14
           + ux * uz * g15 - 4 * uy * uz * g16
           + 0.5 * ux * g17 - ux * g18 + 2 * uz * g21 + 2 * uy * g22)
    g24 = (w[24] / 8 * (-exxyzz + 2 * ux * exyzz + 2 * uz * exxyz + uy * exxzz - ux**2 * eyzz
                        - uz**2 * exxy - 2 * ux * uy * exzz - 2 * uy * uz * exxz
                        - 4 * ux * uz * exyz + uy * uz**2 * exx + ux**2 * uy * ezz
                        + 2 * ux * uz**2 * exy + 2 * ux**2 * uz * eyz + 4 * ux * uy * uz * exz
                        - 4 * rho * ux**2 * uy * uz**2 - 0.5 * ux**2 * uz**2 * sy
                        - uy * (ux * uz**2 * sx + ux**2 * uz * sz))
           + (3 * ux * uz**2 + 2 * ux) * g4 + 6 * ux * uy * uz * g5
           + (3 * ux**2 * uz + 2 * uz) * g6 + (0.75 * uy * uz**2 + 0.5 * uy) * g7
           + (0.75 * uy * uz**2 - 1.5 * ux**2 * uy - 0.5 * uy) * g8
           + (0.75 * uy * uz**2 + 0.75 * ux**2 * uy + uy) * g9 - 3 * ux * uy * g10
           + (-1.5 * ux**2 - 1.5 * uz**2 - 2) * g11
           - 3 * uy * uz * g12 + ux * uy * g13 + (0.5 * ux**2 - 0.5 * uz**2) * g14
           - uy * uz * g15 - 4 * ux * uz * g16
           + 0.5 * uy * g17 + 0.5 * uy * g18 - 0.5 * uy * g19 + 2 * uz * g20 + 2 * ux * g22)
    # reading: the g_16 coefficient of g_25 is printed -6 ux uy; the definition
    # gives -4 ux uy.
    g25 = (w[25] / 8 * (-exxyyz + 2 * ux * exyyz + 2 * uy * exxyz + uz * exxyy - ux**2 * eyyz
                        - uy**2 * exxz - 2 * ux * uz * exyy - 2 * uy * uz * exxy
                        - 4 * ux * uy * exyz + uy**2 * uz * exx + ux**2 * uz * eyy
                        + 2 * ux * uy**2 * exz + 2 * ux**2 * uy * eyz + 4 * ux * uy * uz * exy
                        - 4 * rho * ux**2 * uy**2 * uz - 0.5 * ux**2 * uy**2 * sz
                        - uz * (ux * uy**2 * sx + ux**2 * uy * sy))
           + 6 * ux * uy * uz * g4 + (3 * ux * uy**2 + 2 * ux) * g5
           + (3 * ux**2 * uy + 2 * uy) * g6 + (0.75 * uy**2 * uz - 0.75 * ux**2 * uz) * g7
           + (0.75 * uy**2 * uz + 0.75 * ux**2 * uz + uz) * g8
           + (0.75 * uy**2 * uz + 0.75 * ux**2 * uz + uz) * g9 - 3 * ux * uz * g10
           - 3 * uy * uz * g11 + (-1.5 * ux**2 - 1.5 * uy**2 - 2) * g12
           - ux * uz * g13 - uy * uz * g14 + (0.5 * ux**2 - 0.5 * uy**2) * g15
           - 4 * ux * uy * g16
           + 0.5 * uz * g17 + 0.5 * uz * g18 + 0.5 * uz * g19 + 2 * uy * g20 + 2 * ux * g21)
    g26 = (w[26] / 8 * (-exxyyzz + 2 * (ux * exyyzz + uy * exxyzz + uz * exxyyz)
                        - (ux**2 * eyyzz + uy**2 * exxzz + uz**2 * exxyy)
                        - 4 * (ux * uy * exyzz + ux * uz * exyyz + uy * uz * exxyz)
                        + 2 * (ux**2 * uy * eyzz + ux * uy**2 * exzz + ux**2 * uz * eyyz
                               + ux * uz**2 * exyy + uy**2 * uz * exxz + uy * uz**2 * exxy)
                        + 8 * ux * uy * uz * exyz
                        - (uy**2 * uz**2 * exx + ux**2 * uz**2 * eyy + ux**2 * uy**2 * ezz)
                        - 4 * ux * uy * uz * (uz * exy + uy * exz + ux * eyz)
                        + 5 * rho * ux**2 * uy**2 * uz**2 + kxx * kyy * kzz
                        + ux * uy * uz * (ux * uy * sz + ux * uz * sy + uy * uz * sx))
           + (-4 * ux * uy - 6 * ux * uy * uz**2) * g4 + (-4 * ux * uz - 6 * ux * uy**2 * uz) * g5
           + (-4 * uy * uz - 6 * ux**2 * uy * uz) * g6
           + (0.5 * ux**2 - 0.5 * uy**2 + 0.75 * ux**2 * uz**2 - 0.75 * uy**2 * uz**2) * g7
           + (0.5 * ux**2 + 0.5 * uy**2 - uz**2 - 0.75 * uy**2 * uz**2 - 0.75 * ux**2 * uz**2
              + 1.5 * ux**2 * uy**2) * g8
           + (-ux**2 - uy**2 - uz**2 - 0.75 * ux**2 * uy**2 - 0.75 * ux**2 * uz**2
              - 0.75 * uy**2 * uz**2 - 1) * g9
           + (3 * ux * uy**2 + 3 * ux * uz**2 + 4 * ux) * g10
           + (3 * ux**2 * uy + 3 * uy * uz**2 + 4 * uy) * g11
           + (3 * ux**2 * uz + 3 * uy**2 * uz + 4 * uz) * g12 + (ux * uz**2 - ux * uy**2) * g13
           + (uy * uz**2 - ux**2 * uy) * g14 + (uy**2 * uz - ux**2 * uz) * g15
           + 8 * ux * uy * uz * g16
           + (-0.5 * ux**2 - 0.5 * uy**2 - 0.5 * uz**2 - 1) * g17
           + (ux**2 - 0.5 * uy**2 - 0.5 * uz**2) * g18
           + (0.5 * uy**2 - 0.5 * uz**2) * g19 - 4 * uy * uz * g20 - 4 * ux * uz * g21
           - 4 * ux * uy * g22 + 2 * ux * g23 + 2 * uy * g24 + 2 * uz * g25)
    g = np.zeros_like(f)
    for k, v in enumerate([g4, g5, g6, g7, g8, g9, g10, g11, g12, g13, g14, g15, g16, g17, g18,
                           g19, g20, g21, g22, g23, g24, g25, g26]):
        g[:, 4 + k] = v
    return g, (kxx, kyy, kzz)


def kernels_q15(f, F, om, e):
    """App. G: printed D3Q15 collision kernels g_4..g_14 (used as printed).
    kappa~_xx, kappa~_yy are not printed for D3Q15; they follow from the
    printed moments of the D3Q15 collision kernel (App. G) in the same way as
    the D3Q27 ones of Sec. 7."""
    rho, u = _macro(f, F, e)
    ux, uy, uz = u[:, 0], u[:, 1], u[:, 2]
    kb = raw_moments(f, IDX15)
    sg = raw_source_moments(F, u)
    E = {k: kb[k] + sg[k] for k in kb}
    sx, sy, sz = sg["x"], sg["y"], sg["z"]
    w = om
    exy, exz, eyz, exx, eyy, ezz = E["xy"], E["xz"], E["yz"], E["xx"], E["yy"], E["zz"]
    g4 = w[4] / 8 * (-exy + rho * ux * uy + 0.5 * (sx * uy + sy * ux))
    g5 = w[5] / 8 * (-exz + rho * ux * uz + 0.5 * (sx * uz + sz * ux))
    g6 = w[6] / 8 * (-eyz + rho * uy * uz + 0.5 * (sy * uz + sz * uy))
    g7 = w[7] / 4 * (-(exx - eyy) + rho * (ux**2 - uy**2) + (sx * ux - sy * uy))
    g8 = w[8] / 12 * (-(exx + eyy - 2 * ezz) + rho * (ux**2 + uy**2 - 2 * uz**2)
                      + (sx * ux + sy * uy - 2 * sz * uz))
    g9 = w[9] / 18 * (-(exx + eyy + ezz) + rho * (ux**2 + uy**2 + uz**2)
                      + (sx * ux + sy * uy + sz * uz) + rho)
    g10 = (w[10] / 16 * (-E["xyy"] + 2 * uy * exy + ux * eyy - 2 * rho * ux * uy**2
                         - 0.5 * sx * uy**2 - sy * uy * ux)
           + uy * g4 + 0.125 * ux * (-g7 + g8 + 3 * g9))
    g11 = (w[11] / 16 * (-E["xxy"] + 2 * ux * exy + uy * exx - 2 * rho * ux**2 * uy
                         - 0.5 * sy * ux**2 - sx * ux * uy)
           + ux * g4 + 0.125 * uy * (g7 + g8 + 3 * g9))
    g12 = (w[12] / 16 * (-E["xxz"] + 2 * ux * exz + uz * exx - 2 * rho * ux**2 * uz
                         - 0.5 * sz * ux**2 - sx * ux * uz)
           + ux * g5 + 0.125 * uz * (g7 + g8 + 3 * g9))
    g13 = (w[13] / 8 * (-E["xyz"] + ux * eyz + uy * exz + uz * exy - 2 * rho * ux * uy * uz
                        - 0.5 * (sx * uy * uz + sy * ux * uz + sz * ux * uy))
           + uz * g4 + uy * g5 + ux * g6)
    kxx = exx + 2 * g7 + 2 * g8 + 6 * g9 - rho * ux**2 - F[:, 0] * ux
    kyy = eyy - 2 * g7 + 2 * g8 + 6 * g9 - rho * uy**2 - F[:, 1] * uy
    g14 = (w[14] / 16 * (-E["xxyy"] + 2 * ux * E["xyy"] + 2 * uy * E["xxy"] - ux**2 * eyy
                         - uy**2 * exx - 4 * ux * uy * exy + kxx * kyy + 3 * rho * ux**2 * uy**2
                         + sx * ux * uy**2 + sy * uy * ux**2)
           - 2 * ux * uy * g4 + 0.125 * (ux**2 - uy**2) * g7 + 0.125 * (-ux**2 - uy**2) * g8
           + (0.375 * (-ux**2 - uy**2) - 0.5) * g9 + 2 * ux * g10 + 2 * uy * g11)
    g = np.zeros_like(f)
    for k, v in enumerate([g4, g5, g6, g7, g8, g9, g10, g11, g12, g13, g14]):
        g[:, 4 + k] = v
    return g, (kxx, kyy)
