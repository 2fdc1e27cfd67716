/*
 * lbm.h -- C ABI of the GB300 (sm_103a) central-moment lattice Boltzmann
 * library, liblbm.so.
 *
 * The method is the three-dimensional central-moment LBM with forcing terms
 * of Premnath & Banerjee ("On the three-dimensional central moment lattice
 * Boltzmann method"), on the D3Q27 lattice (Sec. 2-8) and the D3Q15 lattice
 * (App. G).  One time step is the fused collide-and-stream update
 *     f~(x, t)          = f(x, t) + K.g(x, t) + S(x, t)   (Eq. cascadedcollision1)
 *     f(x + e_a, t + 1) = f~_a(x, t)                      (Eq. cascadedstreaming1)
 * where f is the transformed distribution f-bar = f - S/2 of Sec. 4, g the
 * cascaded central-moment collision kernel of Sec. 7 and S the
 * semi-implicit source term of App. E / App. G.
 *
 * Conventions shared by every call:
 *   - Grid: nx * ny * nz cells; cell (x, y, z) has dense index
 *     c = (z * ny + y) * nx + x.  x is always periodic; y and z are periodic
 *     or closed by half-way bounce-back walls (Sec. 9), see LBM_WALL_*.
 *   - Velocity order: the paper's, alpha = 0..Q-1 (Eq. velocityd3qq27 and
 *     the component lists of Sec. 2 for D3Q27; Eq. velocityd3q15 and the
 *     matrix of App. G for D3Q15).
 *   - Dense fields exchanged with the caller are structure-of-arrays:
 *     distributions [Q][nz][ny][nx], vectors [3][nz][ny][nx], scalars
 *     [nz][ny][nx].  Every pointer argument named "device" is memory the
 *     GPU that was current at lbm_create addresses directly: its own device
 *     memory, or page-locked host memory mapped into its address space
 *     (cudaHostAlloc / cudaHostRegister under unified addressing).  The
 *     dense fields of lbm_init_equilibrium, lbm_set_state, lbm_get_state
 *     and lbm_macroscopic may be such host buffers: the kernels then read
 *     or write them across the host link themselves, with no separate copy
 *     (state buffers, force fields and adjoint fields must be device
 *     memory).  "host" is plain host memory.
 *   - Ownership: the caller allocates and frees every device buffer and owns
 *     every stream it passes.  The library allocates only its context, a
 *     small reduction scratch, and for lbm_step a private capture stream and
 *     the CUDA graphs it captures, all released by lbm_destroy.
 *   - Streams: a `void *stream` argument is a cudaStream_t (NULL = the legacy
 *     default stream).  Every call is asynchronous on that stream except
 *     lbm_conservation and lbm_kinetic_energy, which synchronise it.
 *   - Errors: every call returns an lbm_status; nothing throws, aborts or
 *     prints.  Argument errors are detected before any work is enqueued and
 *     leave the context unchanged.  A CUDA launch error is reported as
 *     LBM_ECUDA (the CUDA error string is available from
 *     lbm_last_cuda_error).
 *   - Thread safety: one context must not be used from two host threads at
 *     once; distinct contexts are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LBM_D3Q15 = 15, LBM_D3Q27 = 27 } lbm_lattice;

/* How the two state buffers hold the distributions.  All arithmetic is FP32
 * whatever the storage.  LBM_STORE_F32 keeps f - w_a (the deviation from the
 * lattice weight w_a, the rest state at rho = 1) in FP32; the 16-bit modes
 * keep (f - w_a) / w_a in FP16 or BF16, stochastically rounded by the step
 * (up or down with probability proportional to the distance, from bits
 * hashed out of the values and the cell, so a recomputed step rounds the
 * same way) and rounded to nearest when a state is loaded.  BF16 (8
 * significant bits) stores the populations with one or two nonzero velocity
 * components relative to the linear part of the local equilibrium:
 * (f_a - w_a) / w_a - e_a . J, with J = 3 times the mean velocity of the pair
 * of cells (x even, x + 1) whose collision produced the value; J of every
 * pair is kept in FP32 after the population planes (8 bytes per cell), so
 * a BF16 state buffer is self-contained (see lbm_state_bytes). */
typedef enum { LBM_STORE_F32 = 0, LBM_STORE_F16 = 1, LBM_STORE_BF16 = 2 } lbm_storage;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,       /* bad argument (null pointer, size, rate, alias) */
    LBM_ENOMEM = 2,       /* the library's own scratch could not be allocated */
    LBM_ESTATE = 3,       /* call out of order (e.g. step before bind) */
    LBM_ECUDA = 4,        /* a CUDA call or kernel launch failed */
    LBM_ENONFINITE = 5,   /* a conservation sum is NaN or infinite */
    LBM_EUNSUPPORTED = 6  /* valid request this build does not provide */
} lbm_status;

/* bc_flags of lbm_create: half-way bounce-back walls on the y faces
 * (between y = -1 and 0 and between ny - 1 and ny) and/or the z faces. */
#define LBM_WALL_Y 1u
#define LBM_WALL_Z 2u

/* bc_flags of lbm_create: single-buffer in-place streaming (the "AA"
 * access pattern; not in the paper, which states the update with separate
 * collision and streaming steps, Eqs. cascadedcollision1 and
 * cascadedstreaming1).  The context then works on ONE state buffer:
 * lbm_bind takes f_b = NULL.  Steps alternate between two kernels: the
 * first collides every cell in place and stores its post-collision values
 * in the opposite slots of the same cell; the second reads them from the
 * upstream neighbours, collides and writes the results to the downstream
 * neighbours' slots (bounce-back walls as in the two-buffer scheme).  Every
 * thread reads and writes the same locations, so no second buffer is needed
 * and each step moves the same bytes as a two-buffer step.  The results are
 * bit-identical to the two-buffer scheme.  Requires nx even.
 * lbm_current_state returns NULL and lbm_step_into and lbm_adjoint_step
 * return LBM_EUNSUPPORTED for such a context (their buffers hold two-buffer
 * states). */
#define LBM_INPLACE 4u

/* bc_flags of lbm_create: stochastically rounded FP32 update (FP32 storage
 * only; not with LBM_INPLACE).  Each step computes the collision's change
 * d = f~ - f and stores f + d rounded up or down to FP32 with probability
 * proportional to the distance (the exact sum from an error-free two-sum),
 * instead of to nearest.  Meant for long runs to a steady state on small
 * grids: there round-to-nearest makes the same rounding error at every step
 * and those errors add up in the slowest modes (the grid-convergence study
 * of Sec. 9 stops converging near 3e-4 relative error in FP32); with this
 * flag they average out.  The rounding is a fixed function of the state.
 * It runs the one-cell-per-thread kernel and costs throughput; not in the
 * paper. */
#define LBM_F32_SR 8u

typedef struct lbm_ctx lbm_ctx;

/* Create a solver context for one grid.
 *   lattice  LBM_D3Q27 or LBM_D3Q15.
 *   nx,ny,nz grid size, each >= 1, ny and nz <= 65535, and
 *            nx*ny*nz < 2^31 (one population plane is addressed with 32-bit
 *            offsets; 1024^3 fits).
 *   omega    host, Q relaxation rates omega_beta of the cascade (Sec. 7);
 *            entries 0..3 are ignored (collision invariants), the others
 *            must lie in (0, 2).  omega_4..omega_8 set the shear viscosity
 *            nu = (1/omega - 1/2)/3 (end of Sec. 7; App. G).
 *   force    host, 3 values: the uniform body force F (lattice units); used
 *            when no force field is bound.  NULL means zero.
 *   bc_flags OR of LBM_WALL_Y / LBM_WALL_Z (0: fully periodic), optionally
 *            with LBM_INPLACE (then nx must be even) or LBM_F32_SR (then
 *            storage must be LBM_STORE_F32, and not LBM_INPLACE).
 *   storage  an lbm_storage value.
 *   out      receives the context (set to NULL on error).
 * Errors: LBM_EINVAL, LBM_ENOMEM (context allocation), LBM_ECUDA (no usable
 * device).  The GPU current at this call is the context's device. */
lbm_status lbm_create(lbm_lattice lattice, int nx, int ny, int nz, const double *omega,
                      const double *force, unsigned bc_flags, lbm_storage storage,
                      lbm_ctx **out);

/* Release the context, its reduction scratch, capture stream and CUDA
 * graphs (not the caller's buffers).  Safe on NULL.  Work already enqueued
 * must have completed. */
void lbm_destroy(lbm_ctx *ctx);

/* Size in bytes of each of the two state buffers the caller must provide:
 * Q populations of ny * nz rows of a row pitch >= nx elements (a multiple of
 * 32 elements), in the storage type; for LBM_STORE_BF16 followed by the
 * momentum references (one float4 per pair of cells of the pitched rows,
 * 8 bytes per cell; two such arrays with LBM_INPLACE).  A state is fully
 * described by these bytes: copying them copies the state.  0 for a NULL
 * context. */
size_t lbm_state_bytes(const lbm_ctx *ctx);

/* Row pitch in elements of the state buffers (see lbm_state_bytes). */
int lbm_row_pitch(const lbm_ctx *ctx);

/* Attach the caller's two state buffers (device, lbm_state_bytes each,
 * 256-byte aligned, not overlapping) and an optional per-cell force field
 * force_field (device, FP32 [3][nz][ny][nx], NULL = the uniform force).
 * A context created with LBM_INPLACE takes one buffer: f_b must be NULL.
 * The buffers' contents are undefined until lbm_init_equilibrium or
 * lbm_set_state.  Rebinding is allowed between steps.
 * Errors: LBM_EINVAL (null, misaligned or equal buffers). */
lbm_status lbm_bind(lbm_ctx *ctx, void *f_a, void *f_b, const float *force_field);

/* Replace the uniform body force (host, 3 values; NULL = zero) used by the
 * following steps when no force field is bound.  Takes effect for work
 * enqueued after this call (the value is passed by argument to each launch). */
lbm_status lbm_set_force(lbm_ctx *ctx, const double *force);

/* Replace the per-cell force field (device FP32 [3][nz][ny][nx]; NULL = use
 * the uniform force) for work enqueued after this call; the state is kept. */
lbm_status lbm_set_force_field(lbm_ctx *ctx, const float *force_field);

/* Replace the relaxation rates (host, Q values, as in lbm_create). */
lbm_status lbm_set_omega(lbm_ctx *ctx, const double *omega);

/* Set the state to f = f^at(rho, u) - S(F, u)/2 at every cell: f^at is the
 * attractor state of the collision (the central moments of
 * Eq. transformedcentralmomentattractors: rho, 0, rho/3, ..., with the
 * factorised higher orders) and S the source of App. E / App. G, so that
 * Eqs. densitycalculation and velocitycalculation return rho and u.
 *   rho device FP64 [nz][ny][nx];  u device FP64 [3][nz][ny][nx].
 * The paper does not prescribe an initial state; this is the library's
 * choice.  Errors: LBM_ESTATE (not bound), LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u, void *stream);

/* Load an arbitrary state f (device FP64 [Q][nz][ny][nx], the transformed
 * distributions f-bar at the current time), converting to the storage type.
 * Errors: LBM_ESTATE, LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_set_state(lbm_ctx *ctx, const double *f, void *stream);

/* Read the current state back (device FP64 [Q][nz][ny][nx]). */
lbm_status lbm_get_state(const lbm_ctx *ctx, double *f, void *stream);

/* Advance nsteps >= 0 fused collide-and-stream steps (Eqs. cascadedcollision1
 * and cascadedstreaming1), one kernel launch per step on `stream` (with
 * LBM_INPLACE, alternately the in-place and the neighbour kernel).  Runs of
 * lbm_set_graph_steps steps (32 by default) are launched as one CUDA graph,
 * captured on first use for the current force, rates, buffers and parity
 * and replayed while those stay the same; the rest step by step.  Inside a
 * stream capture of the caller's, every step is launched on its own.
 * Errors: LBM_ESTATE (not bound), LBM_EINVAL (nsteps < 0), LBM_ECUDA. */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps, void *stream);

/* Steps per CUDA graph in lbm_step: an even count >= 2, or 0 to launch every
 * step on its own (graphs cut the host's launch cost, which bounds small
 * grids).  Results do not depend on it.  Not in the paper.
 * Errors: LBM_EINVAL (negative or odd). */
lbm_status lbm_set_graph_steps(lbm_ctx *ctx, int steps);

/* Density and velocity of the current state, Eqs. densitycalculation and
 * velocitycalculation (u includes the +F/2 shift):
 *   rho device FP32 [nz][ny][nx] (may be NULL);  u device FP32 [3][nz][ny][nx]
 *   (may be NULL). */
lbm_status lbm_macroscopic(const lbm_ctx *ctx, float *rho, float *u, void *stream);

/* Global mass and momentum of the current state, sum_x rho and
 * sum_x rho u (with the +F/2 shift): per-cell moments in FP32, sums across
 * cells in FP64 on the GPU (collision invariants, Sec. 4).  out: host, 4 doubles.  Synchronises
 * `stream`.  Deterministic (fixed reduction order).
 * Errors: LBM_ESTATE, LBM_ENOMEM (scratch), LBM_ECUDA, LBM_ENONFINITE (out is
 * still written). */
lbm_status lbm_conservation(lbm_ctx *ctx, double out[4], void *stream);

/* ---- discrete adjoint (D3Q27 and D3Q15; not in the paper: the reverse mode
 * of its update, for gradients with respect to a per-cell body force) --- */

/* Size in bytes of one adjoint field lam: FP32, laid out like an FP32 state
 * buffer (Q population planes of pitched rows; see lbm_state_bytes). */
size_t lbm_adjoint_bytes(const lbm_ctx *ctx);

/* The bound buffer that holds the current state (NULL before a state is
 * set).  Valid until the next lbm_step / lbm_bind; lets a caller checkpoint
 * the state with a device-to-device copy of lbm_state_bytes. */
const void *lbm_current_state(const lbm_ctx *ctx);

/* One collide-and-stream step from the state in f_in to f_out (device,
 * lbm_state_bytes each, 256-byte aligned, not overlapping; any buffers, not
 * only the bound pair, e.g. a checkpoint ring).  The bound pair and the
 * current state are untouched.  Errors: LBM_EINVAL, LBM_EUNSUPPORTED
 * (LBM_INPLACE context), LBM_ECUDA. */
lbm_status lbm_step_into(lbm_ctx *ctx, const void *f_in, void *f_out, void *stream);

/* Adjoint of one step taken from the state f_t (a state buffer holding the
 * state at time t):
 *     lam_out(y) = J_C(f_t(y))^T mu(y),  mu_a(y) = lam_next_a(y + e_a)
 * (lam_next_opp(a)(y) where y + e_a is behind a bounce-back wall), J_C the
 * per-cell Jacobian of the collision, and, when dJdF is not NULL,
 *     dJdF(y) += (dC/dF(y))^T mu(y)
 * (device FP32 [3][nz][ny][nx], accumulated; the force of step t is the
 * bound force field or the uniform force).  lam_next, lam_out: device FP32
 * adjoint fields (lbm_adjoint_bytes, 16-byte aligned, not overlapping: the
 * step reads lam_next at neighbouring cells while it writes lam_out).
 * Errors: LBM_EINVAL, LBM_EUNSUPPORTED (LBM_INPLACE context), LBM_ECUDA. */
lbm_status lbm_adjoint_step(lbm_ctx *ctx, const void *f_t, const float *lam_next,
                            float *lam_out, float *dJdF, void *stream);

/* Kinetic energy J = sum_x rho |u|^2 / 2 of the state in f (a state buffer
 * in the two-buffer layout; NULL = the current state, in either scheme),
 * u with the +F/2 shift; per-cell values in
 * FP32, summed in FP64.  out: host, 1 double.  Synchronises `stream`.
 * Errors: LBM_EINVAL, LBM_ESTATE, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE. */
lbm_status lbm_kinetic_energy(lbm_ctx *ctx, const void *f, double *out, void *stream);

/* Seed of the adjoint of J: lam_out = dJ/df of the state in f (NULL =
 * current), lam_a = u.e_a - |u|^2/2, and, when dJdF is not NULL, the direct
 * term dJdF += u/2.  lam_out: an adjoint field (lbm_adjoint_bytes, 16-byte
 * aligned); dJdF: device FP32 [3][nz][ny][nx], 4-byte aligned, accumulated.
 * Errors: LBM_EINVAL, LBM_ESTATE, LBM_ECUDA. */
lbm_status lbm_kinetic_energy_seed(lbm_ctx *ctx, const void *f, float *lam_out, float *dJdF,
                                   void *stream);

/* Seed of the adjoint of any objective J(rho, u) of the macroscopic fields
 * of the state in f (a two-buffer state buffer; NULL = the current state),
 * given its gradients g_rho = dJ/drho (device FP32 [nz][ny][nx]) and
 * g_u = dJ/du (device FP32 [3][nz][ny][nx]); either may be NULL (zero).
 * With rho and u of Eqs. densitycalculation and velocitycalculation
 * (u = (sum f e + F/2) / rho), d rho/d f_a = 1 and d u_i/d f_a =
 * (e_ai - u_i)/rho, so
 *     lam_out_a(x) = g_rho(x) + sum_i (e_ai - u_i(x)) g_u_i(x) / rho(x),
 * and, when dJdF is not NULL, the direct term dJdF_i += g_u_i / (2 rho).
 * lam_out: an adjoint field (lbm_adjoint_bytes, 16-byte aligned).  Not in
 * the paper (reverse mode of its output step).
 * Errors: LBM_EINVAL, LBM_ESTATE, LBM_ECUDA. */
lbm_status lbm_macroscopic_seed(lbm_ctx *ctx, const void *f, const float *g_rho,
                                const float *g_u, float *lam_out, float *dJdF, void *stream);

/* Conservation sums for callers that cannot let the library allocate device
 * memory (the paper has no counterpart; this is a library service).  Same
 * sums as lbm_conservation, but asynchronous, into a caller buffer, and with
 * no cudaMalloc or cudaFree: the per-row partial sums live in a fixed array
 * inside the library, 2 MiB per GPU, held by every GPU that loads the
 * library until the process exits.
 *   out  4 doubles (8-byte aligned) that the context's GPU can write:
 *        its own device memory, managed memory, or page-locked host memory
 *        mapped into its address space (anything else, e.g. a plain host
 *        array, is refused with LBM_EINVAL before any launch):
 *        sum_x (rho - 1), then sum_x rho u_x, rho u_y, rho u_z.  Note: the
 *        first value is the mass minus the cell count nx*ny*nz (the FP64
 *        sum of the density deviations, without the large constant).
 * Limit: ny * nz <= 65536 (one partial record per (y, z) row); larger grids
 * return LBM_EINVAL.  The context's device must be current (LBM_ESTATE
 * otherwise).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for the life of the process;
 * make that first call before any stream capture, and make no call after a
 * cudaDeviceReset of that device (the kept address would no longer be
 * valid).  All calls share the array: calls whose work overlaps on the GPU
 * race.  Errors: LBM_EINVAL, LBM_ESTATE, LBM_ECUDA, LBM_EUNSUPPORTED (device
 * index >= 64). */
lbm_status lbm_conservation_noalloc(lbm_ctx *ctx, double *out, void *stream);

/* Human-readable name of a status code (static string). */
const char *lbm_status_string(lbm_status status);

/* CUDA error string of the context's last LBM_ECUDA (static string; "" if none). */
const char *lbm_last_cuda_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
