/* A plain C client of liblbm.so (no Python, no PyTorch): a periodic D3Q27
 * box at rest under a uniform body force.  It owns its device buffers
 * (cudaMalloc), drives the library through include/lbm.h only, and prints
 * the FP64 conservation sums after each run of steps.  The initial state
 * has u = 0 (velocity with the +F/2 shift of Eq. velocitycalculation) and
 * every step adds F to the momentum of every cell, so sum_x rho u = N F t,
 * and the mass stays N.
 *
 * usage: momentum_box [nx ny nz steps]    output: one line per run of steps
 *   "t mass momentum_x momentum_y momentum_z"                              */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "lbm.h"

#define CHECK(call)                                                                  \
    do {                                                                             \
        lbm_status st_ = (call);                                                     \
        if (st_ != LBM_OK) {                                                         \
            fprintf(stderr, "%s: %s\n", #call, lbm_status_string(st_));              \
            return 1;                                                                \
        }                                                                            \
    } while (0)

int main(int argc, char **argv) {
    int nx = 16, ny = 16, nz = 16, steps = 100;
    if (argc == 5) {
        nx = atoi(argv[1]);
        ny = atoi(argv[2]);
        nz = atoi(argv[3]);
        steps = atoi(argv[4]);
    }
    const size_t n = (size_t)nx * ny * nz;
    double omega[27];
    for (int b = 0; b < 27; ++b) omega[b] = (b >= 4 && b <= 8) ? 1.0 / 0.6 : 1.0;
    const double force[3] = {1e-5, -2e-5, 3e-5};
    if (cudaSetDevice(0) != cudaSuccess) return 2;

    lbm_ctx *ctx = NULL;
    CHECK(lbm_create(LBM_D3Q27, nx, ny, nz, omega, force, 0u, LBM_STORE_F32, &ctx));
    /* a call out of order is reported, not fatal */
    if (lbm_step(ctx, 1, NULL) != LBM_ESTATE) return 3;

    void *fa = NULL, *fb = NULL;
    double *rho = NULL, *u = NULL;
    const size_t bytes = lbm_state_bytes(ctx);
    if (cudaMalloc(&fa, bytes) || cudaMalloc(&fb, bytes) ||
        cudaMalloc((void **)&rho, n * sizeof(double)) ||
        cudaMalloc((void **)&u, 3 * n * sizeof(double)))
        return 4;
    double *h = (double *)calloc(3 * n, sizeof(double));
    if (!h) return 5;
    for (size_t i = 0; i < n; ++i) h[i] = 1.0;
    cudaMemcpy(rho, h, n * sizeof(double), cudaMemcpyHostToDevice);
    for (size_t i = 0; i < n; ++i) h[i] = 0.0;
    cudaMemcpy(u, h, 3 * n * sizeof(double), cudaMemcpyHostToDevice);

    CHECK(lbm_bind(ctx, fa, fb, NULL));
    CHECK(lbm_init_equilibrium(ctx, rho, u, NULL));
    int t = 0;
    for (int run = 0; run < 3; ++run) {
        double out[4];
        CHECK(lbm_conservation(ctx, out, NULL));
        printf("%d %.17g %.17g %.17g %.17g\n", t, out[0], out[1], out[2], out[3]);
        CHECK(lbm_step(ctx, steps, NULL));
        t += steps;
    }
    double out[4];
    CHECK(lbm_conservation(ctx, out, NULL));
    printf("%d %.17g %.17g %.17g %.17g\n", t, out[0], out[1], out[2], out[3]);

    lbm_destroy(ctx);
    cudaFree(fa);
    cudaFree(fb);
    cudaFree(rho);
    cudaFree(u);
    free(h);
    return 0;
}
