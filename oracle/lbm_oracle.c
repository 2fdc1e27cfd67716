/*
 * FP64 CPU oracle of the three-dimensional central-moment lattice Boltzmann
 * method with forcing terms (Premnath & Banerjee, "On the three-dimensional
 * central moment lattice Boltzmann method"), for the D3Q27 and D3Q15 lattices.
 *
 * TEST INFRASTRUCTURE.  This library is the parity reference of the CUDA path
 * and the timed CPU baseline.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no source,
 * header, table or helper with the CUDA path, and the product never calls it.
 *
 * Every step is the plain definition, written out, with no fusion, blocking
 * or reordering beyond what the paper states:
 *   - velocity sets and their order: Sec. 2 (Eq. velocityd3qq27 and the
 *     component lists of the conserved basis vectors), App. G (D3Q15);
 *   - moment basis K as polynomials of the particle velocity: Sec. 2 (D3Q27),
 *     App. G (D3Q15); the matrix K[alpha][beta] = K_beta(e_alpha) and
 *     D = diag(<K_beta|K_beta>);
 *   - density and velocity with the +F/2 shift: Eqs. densitycalculation and
 *     velocitycalculation (Sec. 6);
 *   - raw source moments by the binomial theorem from the central source
 *     moments (0, F, 0, ...): Eq. forcingaliased, Eq. discretecentralsources,
 *     App. C; projections m^s_beta = <K_beta|S>: App. D / App. G;
 *   - source in velocity space by exact inversion S = K D^-1 m^s
 *     (Eq. sourceformulation1 and the orthogonality of K; App. E);
 *   - collision kernel by the cascade of Sec. 7: for beta = 4..Q-1 in order,
 *     the central moment P_beta of the post-collision state is relaxed toward
 *     its attractor (Eq. transformedcentralmomentattractors) with omega_beta
 *     applied only to the terms that do not yet contain g_gamma, gamma < beta;
 *     g_0..g_3 = 0 (collision invariants);
 *   - post-collision state f~ = f + K.g + S: Eq. cascadedcollision1, Sec. 8;
 *   - streaming f(x + e_alpha, t + 1) = f~(x, t): Eq. cascadedstreaming1,
 *     with half-way bounce-back at walls (Sec. 9).
 *
 * The same collision source is compiled twice, once in double and once in
 * double complex; the complex copy gives exact per-cell Jacobians by the
 * complex-step method (derivative = Im f(x + i h) / h), which the oracle
 * adjoint uses.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 27
#define ORACLE_WALL_Y 1u
#define ORACLE_WALL_Z 2u

typedef struct { double c; int m, n, p; } mono_t;      /* c * x^m y^n z^p */
typedef struct { int nt; mono_t t[8]; } poly_t;

#define T(c, m, n, p) { (c), (m), (n), (p) }

/* Sec. 2: orthogonal basis of the D3Q27 lattice, K_0..K_26, written out as
 * polynomials of (e_x, e_y, e_z). */
static const poly_t K27[27] = {
    {1, {T(1, 0, 0, 0)}},
    {1, {T(1, 1, 0, 0)}},
    {1, {T(1, 0, 1, 0)}},
    {1, {T(1, 0, 0, 1)}},
    {1, {T(1, 1, 1, 0)}},
    {1, {T(1, 1, 0, 1)}},
    {1, {T(1, 0, 1, 1)}},
    {2, {T(1, 2, 0, 0), T(-1, 0, 2, 0)}},
    {3, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(-2, 0, 0, 2)}},
    {4, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(1, 0, 0, 2), T(-2, 0, 0, 0)}},
    {3, {T(3, 1, 2, 0), T(3, 1, 0, 2), T(-4, 1, 0, 0)}},
    {3, {T(3, 2, 1, 0), T(3, 0, 1, 2), T(-4, 0, 1, 0)}},
    {3, {T(3, 2, 0, 1), T(3, 0, 2, 1), T(-4, 0, 0, 1)}},
    {2, {T(1, 1, 2, 0), T(-1, 1, 0, 2)}},
    {2, {T(1, 2, 1, 0), T(-1, 0, 1, 2)}},
    {2, {T(1, 2, 0, 1), T(-1, 0, 2, 1)}},
    {1, {T(1, 1, 1, 1)}},
    {7, {T(3, 2, 2, 0), T(3, 2, 0, 2), T(3, 0, 2, 2), T(-4, 2, 0, 0), T(-4, 0, 2, 0),
         T(-4, 0, 0, 2), T(4, 0, 0, 0)}},
    {6, {T(3, 2, 2, 0), T(3, 2, 0, 2), T(-6, 0, 2, 2), T(-4, 2, 0, 0), T(2, 0, 2, 0),
         T(2, 0, 0, 2)}},
    {4, {T(3, 2, 2, 0), T(-3, 2, 0, 2), T(-2, 0, 2, 0), T(2, 0, 0, 2)}},
    {2, {T(3, 2, 1, 1), T(-2, 0, 1, 1)}},
    {2, {T(3, 1, 2, 1), T(-2, 1, 0, 1)}},
    {2, {T(3, 1, 1, 2), T(-2, 1, 1, 0)}},
    {4, {T(9, 1, 2, 2), T(-6, 1, 2, 0), T(-6, 1, 0, 2), T(4, 1, 0, 0)}},
    {4, {T(9, 2, 1, 2), T(-6, 2, 1, 0), T(-6, 0, 1, 2), T(4, 0, 1, 0)}},
    {4, {T(9, 2, 2, 1), T(-6, 2, 0, 1), T(-6, 0, 2, 1), T(4, 0, 0, 1)}},
    {8, {T(27, 2, 2, 2), T(-18, 2, 2, 0), T(-18, 2, 0, 2), T(-18, 0, 2, 2), T(12, 2, 0, 0),
         T(12, 0, 2, 0), T(12, 0, 0, 2), T(-8, 0, 0, 0)}},
};

/* Sec. 7: the central moment whose post-collision value defines g_beta on
 * D3Q27 (the bracket of each printed kernel, with the k_beta of App. F as its
 * normalisation).  Entries 0..3 are the conserved moments. */
static const poly_t P27[27] = {
    {1, {T(1, 0, 0, 0)}},
    {1, {T(1, 1, 0, 0)}},
    {1, {T(1, 0, 1, 0)}},
    {1, {T(1, 0, 0, 1)}},
    {1, {T(1, 1, 1, 0)}},
    {1, {T(1, 1, 0, 1)}},
    {1, {T(1, 0, 1, 1)}},
    {2, {T(1, 2, 0, 0), T(-1, 0, 2, 0)}},
    {3, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(-2, 0, 0, 2)}},
    {3, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(1, 0, 0, 2)}},
    {2, {T(1, 1, 2, 0), T(1, 1, 0, 2)}},
    {2, {T(1, 2, 1, 0), T(1, 0, 1, 2)}},
    {2, {T(1, 2, 0, 1), T(1, 0, 2, 1)}},
    {2, {T(1, 1, 2, 0), T(-1, 1, 0, 2)}},
    {2, {T(1, 2, 1, 0), T(-1, 0, 1, 2)}},
    {2, {T(1, 2, 0, 1), T(-1, 0, 2, 1)}},
    {1, {T(1, 1, 1, 1)}},
    {3, {T(1, 2, 2, 0), T(1, 2, 0, 2), T(1, 0, 2, 2)}},
    {3, {T(1, 2, 2, 0), T(1, 2, 0, 2), T(-2, 0, 2, 2)}},
    {2, {T(1, 2, 2, 0), T(-1, 2, 0, 2)}},
    {1, {T(1, 2, 1, 1)}},
    {1, {T(1, 1, 2, 1)}},
    {1, {T(1, 1, 1, 2)}},
    {1, {T(1, 1, 2, 2)}},
    {1, {T(1, 2, 1, 2)}},
    {1, {T(1, 2, 2, 1)}},
    {1, {T(1, 2, 2, 2)}},
};

/* App. G: orthogonal basis of the D3Q15 lattice. */
static const poly_t K15[15] = {
    {1, {T(1, 0, 0, 0)}},
    {1, {T(1, 1, 0, 0)}},
    {1, {T(1, 0, 1, 0)}},
    {1, {T(1, 0, 0, 1)}},
    {1, {T(1, 1, 1, 0)}},
    {1, {T(1, 1, 0, 1)}},
    {1, {T(1, 0, 1, 1)}},
    {2, {T(1, 2, 0, 0), T(-1, 0, 2, 0)}},
    {3, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(-2, 0, 0, 2)}},
    {4, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(1, 0, 0, 2), T(-2, 0, 0, 0)}},
    {4, {T(5, 3, 0, 0), T(5, 1, 2, 0), T(5, 1, 0, 2), T(-13, 1, 0, 0)}},
    {4, {T(5, 2, 1, 0), T(5, 0, 3, 0), T(5, 0, 1, 2), T(-13, 0, 1, 0)}},
    {4, {T(5, 2, 0, 1), T(5, 0, 2, 1), T(5, 0, 0, 3), T(-13, 0, 0, 1)}},
    {1, {T(1, 1, 1, 1)}},
    {7, {T(30, 2, 2, 0), T(30, 2, 0, 2), T(30, 0, 2, 2), T(-40, 2, 0, 0), T(-40, 0, 2, 0),
         T(-40, 0, 0, 2), T(32, 0, 0, 0)}},
};

/* App. G: the central moment relaxed by each D3Q15 kernel g_beta (bracket of
 * each printed kernel). */
static const poly_t P15[15] = {
    {1, {T(1, 0, 0, 0)}},
    {1, {T(1, 1, 0, 0)}},
    {1, {T(1, 0, 1, 0)}},
    {1, {T(1, 0, 0, 1)}},
    {1, {T(1, 1, 1, 0)}},
    {1, {T(1, 1, 0, 1)}},
    {1, {T(1, 0, 1, 1)}},
    {2, {T(1, 2, 0, 0), T(-1, 0, 2, 0)}},
    {3, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(-2, 0, 0, 2)}},
    {3, {T(1, 2, 0, 0), T(1, 0, 2, 0), T(1, 0, 0, 2)}},
    {1, {T(1, 1, 2, 0)}},
    {1, {T(1, 2, 1, 0)}},
    {1, {T(1, 2, 0, 1)}},
    {1, {T(1, 1, 1, 1)}},
    {1, {T(1, 2, 2, 0)}},
};

/* Sec. 2: D3Q27 particle velocities in the paper's order (alpha = 0..26). */
static const int E27[27][3] = {
    {0, 0, 0},   {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, 1, 0}, {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},   {-1, 0, 1},  {1, 0, -1},
    {-1, 0, -1}, {0, 1, 1},  {0, -1, 1},  {0, 1, -1},  {0, -1, -1}, {1, 1, 1},   {-1, 1, 1},
    {1, -1, 1},  {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1},
};

/* App. G: D3Q15 particle velocities in the paper's order (alpha = 0..14). */
static const int E15[15][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 1},  {-1, 1, 1},  {1, -1, 1},  {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1},
    {-1, -1, -1},
};

typedef struct {
    int Q;
    int e[QMAX][3];
    const poly_t *K;
    const poly_t *P;
    double Kmat[QMAX][QMAX]; /* Kmat[alpha][beta] = K_beta(e_alpha) */
    double D[QMAX];          /* <K_beta|K_beta> */
    int opp[QMAX];           /* e_opp[alpha] = -e_alpha */
} lattice_t;

static double ipow_d(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

static double poly_eval_d(const poly_t *P, double x, double y, double z) {
    double s = 0.0;
    for (int t = 0; t < P->nt; ++t)
        s += P->t[t].c * ipow_d(x, P->t[t].m) * ipow_d(y, P->t[t].n) * ipow_d(z, P->t[t].p);
    return s;
}

static int lattice_init(lattice_t *L, int Q) {
    if (Q == 27) {
        L->K = K27;
        L->P = P27;
        memcpy(L->e, E27, sizeof(E27));
    } else if (Q == 15) {
        L->K = K15;
        L->P = P15;
        memcpy(L->e, E15, sizeof(E15));
    } else {
        return -1;
    }
    L->Q = Q;
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            L->Kmat[a][b] = poly_eval_d(&L->K[b], L->e[a][0], L->e[a][1], L->e[a][2]);
    for (int b = 0; b < Q; ++b) {
        double s = 0.0;
        for (int a = 0; a < Q; ++a) s += L->Kmat[a][b] * L->Kmat[a][b];
        L->D[b] = s;
    }
    for (int a = 0; a < Q; ++a) {
        L->opp[a] = -1;
        for (int b = 0; b < Q; ++b)
            if (L->e[b][0] == -L->e[a][0] && L->e[b][1] == -L->e[a][1] &&
                L->e[b][2] == -L->e[a][2])
                L->opp[a] = b;
    }
    return 0;
}

/* binomial coefficient C(n, k) for the small n of the binomial theorem */
static double binom_small(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* ---- the collision, compiled for real and for complex arithmetic ---- */
#define REAL double
#define FN(name) name##_r
#include "oracle_collide.inc"
#undef REAL
#undef FN

#define REAL double complex
#define FN(name) name##_c
#include "oracle_collide.inc"
#undef REAL
#undef FN

/* ------------------------------------------------------------------ */
/* exported API (ctypes); every array is C-contiguous FP64             */
/* ------------------------------------------------------------------ */

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Tables of the lattice: e[Q][3], K[Q][Q] (K[alpha][beta] = K_beta(e_alpha)),
 * D[Q], and the central-moment polynomials P_beta evaluated at d = e_alpha
 * (u = 0) in Pmat[beta][alpha]. */
int oracle_lattice(int Q, int *e, double *K, double *D, double *Pmat) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    for (int a = 0; a < Q; ++a)
        for (int i = 0; i < 3; ++i) e[3 * a + i] = L.e[a][i];
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) K[a * Q + b] = L.Kmat[a][b];
    for (int b = 0; b < Q; ++b) D[b] = L.D[b];
    if (Pmat)
        for (int b = 0; b < Q; ++b)
            for (int a = 0; a < Q; ++a)
                Pmat[b * Q + a] = poly_eval_d(&L.P[b], L.e[a][0], L.e[a][1], L.e[a][2]);
    return 0;
}

/* Collision of n independent cells.  f, out, g, S: [n][Q]; F: [n][3].
 * g and S (may be NULL) receive the collision kernel g_beta and the source S. */
int oracle_collide(int Q, long n, const double *f, const double *F, const double *omega,
                   double *out, double *g, double *S, double *A, int nthreads) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        collide_r(&L, f + c * Q, F + 3 * c, omega, out + c * Q, g ? g + c * Q : NULL,
                  S ? S + c * Q : NULL, A ? A + c * Q * Q : NULL);
    }
    return 0;
}

/* Source term S(F, u) of App. E for n cells: u, F [n][3], S [n][Q]. */
int oracle_source(int Q, long n, const double *u, const double *F, double *S) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    for (long c = 0; c < n; ++c) source_r(&L, u + 3 * c, F + 3 * c, S + c * Q);
    return 0;
}

/* Jacobian of the collision of n cells by the complex step:
 * J[c][alpha][k] = d out_alpha / d x_k, x = (f_0..f_{Q-1}, F_x, F_y, F_z). */
int oracle_collide_jacobian(int Q, long n, const double *f, const double *F,
                            const double *omega, double *J, int nthreads) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    const double hstep = 1e-30;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        double complex fc[QMAX], Fc[3], oc[QMAX];
        for (int k = 0; k < Q + 3; ++k) {
            for (int a = 0; a < Q; ++a) fc[a] = f[c * Q + a];
            for (int i = 0; i < 3; ++i) Fc[i] = F[3 * c + i];
            if (k < Q)
                fc[k] += I * hstep;
            else
                Fc[k - Q] += I * hstep;
            collide_c(&L, fc, Fc, omega, oc, NULL, NULL, NULL);
            for (int a = 0; a < Q; ++a) J[(c * Q + a) * (Q + 3) + k] = cimag(oc[a]) / hstep;
        }
    }
    return 0;
}

static long cell_index(int x, int y, int z, int nx, int ny) {
    return ((long)z * ny + y) * nx + x;
}

/* Target of population alpha leaving cell (x, y, z), Eq. cascadedstreaming1.
 * Returns the target cell, or -1 when the link crosses a wall (half-way
 * bounce-back: the population comes back to its own cell reversed). */
static long stream_target(const lattice_t *L, int a, int x, int y, int z, int nx, int ny,
                          int nz, unsigned bc) {
    int tx = x + L->e[a][0], ty = y + L->e[a][1], tz = z + L->e[a][2];
    tx = (tx + nx) % nx;
    if (ty < 0 || ty >= ny) {
        if (bc & ORACLE_WALL_Y) return -1;
        ty = (ty + ny) % ny;
    }
    if (tz < 0 || tz >= nz) {
        if (bc & ORACLE_WALL_Z) return -1;
        tz = (tz + nz) % nz;
    }
    return cell_index(tx, ty, tz, nx, ny);
}

/* nsteps collide-and-stream steps.  f, fout: [Q][nz][ny][nx] (SoA, x fastest).
 * Ffield: [3][N] per-cell force, or NULL to use the uniform Funi[3].
 * f and fout may be the same array. */
int oracle_run(int Q, int nx, int ny, int nz, unsigned bc, const double *f,
               const double *Ffield, const double *Funi, const double *omega, int nsteps,
               double *fout, int nthreads) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    if (nx <= 0 || ny <= 0 || nz <= 0 || nsteps < 0) return -2;
    const long N = (long)nx * ny * nz;
    double *cur = malloc(sizeof(double) * Q * N);
    double *post = malloc(sizeof(double) * Q * N);
    if (!cur || !post) {
        free(cur);
        free(post);
        return -3;
    }
    memcpy(cur, f, sizeof(double) * Q * N);
    set_threads(nthreads);
    for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) {
            double fc[QMAX], Fc[3], oc[QMAX];
            for (int a = 0; a < Q; ++a) fc[a] = cur[a * N + c];
            for (int i = 0; i < 3; ++i) Fc[i] = Ffield ? Ffield[i * N + c] : Funi[i];
            collide_r(&L, fc, Fc, omega, oc, NULL, NULL, NULL);
            for (int a = 0; a < Q; ++a) post[a * N + c] = oc[a];
        }
        /* streaming, written as the push of Eq. cascadedstreaming1 */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    long c = cell_index(x, y, z, nx, ny);
                    for (int a = 0; a < Q; ++a) {
                        long t = stream_target(&L, a, x, y, z, nx, ny, nz, bc);
                        if (t >= 0)
                            cur[a * N + t] = post[a * N + c];
                        else
                            cur[L.opp[a] * N + c] = post[a * N + c];
                    }
                }
    }
    memcpy(fout, cur, sizeof(double) * Q * N);
    free(cur);
    free(post);
    return 0;
}

/* Density and velocity of a state, Eqs. densitycalculation and
 * velocitycalculation: rho [N], u [3][N]. */
int oracle_macroscopic(int Q, long N, const double *f, const double *Ffield,
                       const double *Funi, double *rho, double *u) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    for (long c = 0; c < N; ++c) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < Q; ++a) {
            r += f[a * N + c];
            for (int i = 0; i < 3; ++i) j[i] += f[a * N + c] * L.e[a][i];
        }
        rho[c] = r;
        for (int i = 0; i < 3; ++i) {
            double Fi = Ffield ? Ffield[i * N + c] : Funi[i];
            u[i * N + c] = (j[i] + 0.5 * Fi) / r;
        }
    }
    return 0;
}

/* Initial state for given density and velocity fields (not specified by the
 * paper): the collision's own attractor state f^at(rho, u), reached by one
 * collision with every omega_beta = 1 and no force from any state of that mass
 * and momentum, minus half the source, f = f^at - S/2 (the transformation of
 * Sec. 4), so that Eqs. densitycalculation and velocitycalculation give back
 * rho and u.  rho [N], u [3][N], Ffield [3][N] or NULL (then Funi), f [Q][N]. */
int oracle_equilibrium(int Q, long N, const double *rho, const double *u,
                       const double *Ffield, const double *Funi, double *f) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    double ones[QMAX], zero3[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < Q; ++b) ones[b] = 1.0;
    double s = 0.0; /* sum_alpha e_alpha_x^2 */
    for (int a = 0; a < Q; ++a) s += L.e[a][0] * L.e[a][0];
    for (long c = 0; c < N; ++c) {
        double guess[QMAX], at[QMAX], S[QMAX], uc[3], Fc[3];
        for (int i = 0; i < 3; ++i) {
            uc[i] = u[i * N + c];
            Fc[i] = Ffield ? Ffield[i * N + c] : Funi[i];
        }
        for (int a = 0; a < Q; ++a) {
            double eu = L.e[a][0] * uc[0] + L.e[a][1] * uc[1] + L.e[a][2] * uc[2];
            guess[a] = rho[c] / Q + rho[c] * eu / s;
        }
        collide_r(&L, guess, zero3, ones, at, NULL, NULL, NULL);
        source_r(&L, uc, Fc, S);
        for (int a = 0; a < Q; ++a) f[a * N + c] = at[a] - 0.5 * S[a];
    }
    return 0;
}

/* One step of the discrete adjoint of oracle_run (one collide-and-stream step
 * from state f).  Given lam_next = dJ/df at t+1 ([Q][N]), returns
 * lam = dJ/df at t ([Q][N]) and adds dJ/dF(x) to gF ([3][N], NULL to skip).
 * Each cell's Jacobian comes from oracle_collide_jacobian's complex step. */
int oracle_adjoint_step(int Q, int nx, int ny, int nz, unsigned bc, const double *f,
                        const double *Ffield, const double *Funi, const double *omega,
                        const double *lam_next, double *lam, double *gF, int nthreads) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    const long N = (long)nx * ny * nz;
    const double hstep = 1e-30;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        double mu[QMAX];
        /* transpose of the streaming: where did each post-collision value go */
        for (int a = 0; a < Q; ++a) {
            long t = stream_target(&L, a, x, y, z, nx, ny, nz, bc);
            mu[a] = (t >= 0) ? lam_next[a * N + t] : lam_next[L.opp[a] * N + c];
        }
        double complex fc[QMAX], Fc[3], oc[QMAX];
        for (int k = 0; k < Q + 3; ++k) {
            for (int a = 0; a < Q; ++a) fc[a] = f[a * N + c];
            for (int i = 0; i < 3; ++i) Fc[i] = Ffield ? Ffield[i * N + c] : Funi[i];
            if (k < Q)
                fc[k] += I * hstep;
            else
                Fc[k - Q] += I * hstep;
            collide_c(&L, fc, Fc, omega, oc, NULL, NULL, NULL);
            double acc = 0.0;
            for (int a = 0; a < Q; ++a) acc += mu[a] * (cimag(oc[a]) / hstep);
            if (k < Q)
                lam[k * N + c] = acc;
            else if (gF)
                gF[(k - Q) * N + c] += acc;
        }
    }
    return 0;
}
