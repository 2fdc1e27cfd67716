// Reverse mode of the D3Q27 collision (collide_q27.cuh), written by hand.
//
// For one cell, the collision maps the pre-collision deviations f and the
// body force F to the post-collision deviations
//     out = Inv(u) Relax(Shift(u) Sums(f) + sigma(F), u, drho),
//     u   = (j + F/2) / rho,
// with Sums the raw-moment sums, Shift(u) the binomial shift to central
// moments, sigma(F) the central source moments, Relax the cascade and Inv(u)
// the way back.  Given the adjoint mu of `out`, adjoint27 returns
// lam = (d out / d f)^T mu and Fbar = (d out / d F)^T mu.
//
// The u-derivatives of the shifts need no stored intermediates:
//   d/du_x Shift(u) R   = -N_x Shift(u) R,   (N_x K)[m][n][p] = m K[m-1][n][p]
//   d/du_x Inv(u) Dt    =  Inv(u) N_x Dt,
// (the derivative of sum f (e - u)^m is -m sum f (e - u)^(m-1); keeping the
// central moments Dt fixed while u moves adds m du Dt[m-1] to the central
// moments about the old u).  So the reverse only keeps, per cell, the
// pre-source central moments K and the post-collision moments Dt.
#pragma once

#include "collide_q27.cuh"

namespace lbm {

// transpose of dist_from_central: (abar, bbar, cbar) -> (k0bar, k1bar, k2bar)
__device__ __forceinline__ void inv_line_T(float u, float &a, float &b, float &c) {
    const float P = 0.5f * (a + c) - b;
    const float s = 0.5f * (c - a);
    const float k2 = P;
    const float k1 = fmaf(2.0f * u, P, s);
    const float k0 = fmaf(u, fmaf(u, P, s), b);
    a = k0;
    b = k1;
    c = k2;
}

// transpose of central_from_sums: (k0bar, k1bar, k2bar) -> (s0bar, s1bar, s2bar)
__device__ __forceinline__ void shift_line_T(float u, float &k0, float &k1, float &k2) {
    const float s0 = fmaf(u, fmaf(u, k2, -k1), k0);  // k0 - u k1 + u^2 k2
    const float s1 = fmaf(-2.0f * u, k2, k1);
    k0 = s0;
    k1 = s1;
}

// transpose of sums: (s0bar, s1bar, s2bar) -> (abar, bbar, cbar)
__device__ __forceinline__ void sums_line_T(float &s0, float &s1, float &s2) {
    const float a = s0 - s1 + s2;
    const float c = s0 + s1 + s2;
    const float b = s0;
    s0 = a;
    s1 = b;
    s2 = c;
}

// <Dbar, N_x D> etc.: sum over lines of Dbar[1] D[0] + 2 Dbar[2] D[1]
__device__ __forceinline__ void shift_u_terms(const float (&Db)[3][3][3], const float (&D)[3][3][3],
                                              float &gx, float &gy, float &gz) {
    gx = gy = gz = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            gx = fmaf(Db[1][a][b], D[0][a][b], fmaf(2.0f * Db[2][a][b], D[1][a][b], gx));
            gy = fmaf(Db[a][1][b], D[a][0][b], fmaf(2.0f * Db[a][2][b], D[a][1][b], gy));
            gz = fmaf(Db[a][b][1], D[a][b][0], fmaf(2.0f * Db[a][b][2], D[a][b][1], gz));
        }
}

// Reverse of relax27.  Dt: post-collision moments (forward output); Db: on
// input the adjoint of Dt, on output the adjoint of the pre-relaxation D.
// Accumulates the adjoints of u and drho.
__device__ __forceinline__ void relax27_T(const float (&Dt)[3][3][3], float (&Db)[3][3][3],
                                          float ux, float uy, float uz, const Rates27<float> &r,
                                          float &gux, float &guy, float &guz, float &gdrho) {
    const float third = 1.0f / 3.0f;
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const float Kwx = third + ux2, Kwy = third + uy2, Kwz = third + uz2;
    const float dxx = Dt[2][0][0], dyy = Dt[0][2][0], dzz = Dt[0][0][2];
    float gKx = 0.0f, gKy = 0.0f, gKz = 0.0f;        // adjoints of Kw_i
    float gdx = Db[2][0][0], gdy = Db[0][2][0], gdz = Db[0][0][2];  // of dxx, dyy, dzz

    // order 6: dK = kt_x kt_y kt_z - Kw_x Kw_y Kw_z
    {
        const float ktx = Kwx + dxx, kty = Kwy + dyy, ktz = Kwz + dzz;
        const float g = Db[2][2][2];
        Db[2][2][2] = r.omw[26] * g;
        const float gK = r.w[26] * g;
        gdx = fmaf(kty * ktz, gK, gdx);
        gdy = fmaf(ktx * ktz, gK, gdy);
        gdz = fmaf(ktx * kty, gK, gdz);
        // kt_y kt_z - Kw_y Kw_z etc., in the cancellation-free form
        gKx = fmaf(fmaf(Kwy, dzz, fmaf(Kwz, dyy, dyy * dzz)), gK, gKx);
        gKy = fmaf(fmaf(Kwx, dzz, fmaf(Kwz, dxx, dxx * dzz)), gK, gKy);
        gKz = fmaf(fmaf(Kwx, dyy, fmaf(Kwy, dxx, dxx * dyy)), gK, gKz);
    }
    // order 5
    {
        float g = Db[1][2][2];
        Db[1][2][2] = r.omw[23] * g;
        g *= r.w[23];
        gux = fmaf(Kwy * Kwz, g, gux);
        gKy = fmaf(ux * Kwz, g, gKy);
        gKz = fmaf(ux * Kwy, g, gKz);
        g = Db[2][1][2];
        Db[2][1][2] = r.omw[24] * g;
        g *= r.w[24];
        guy = fmaf(Kwx * Kwz, g, guy);
        gKx = fmaf(uy * Kwz, g, gKx);
        gKz = fmaf(uy * Kwx, g, gKz);
        g = Db[2][2][1];
        Db[2][2][1] = r.omw[25] * g;
        g *= r.w[25];
        guz = fmaf(Kwx * Kwy, g, guz);
        gKx = fmaf(uz * Kwy, g, gKx);
        gKy = fmaf(uz * Kwx, g, gKy);
    }
    // order 4, mixed: D~ = omw D + nw Kw_i u_j u_k
    {
        float g = Db[2][1][1];
        Db[2][1][1] = r.omw[20] * g;
        g *= r.nw[20];
        gKx = fmaf(uy * uz, g, gKx);
        guy = fmaf(Kwx * uz, g, guy);
        guz = fmaf(Kwx * uy, g, guz);
        g = Db[1][2][1];
        Db[1][2][1] = r.omw[21] * g;
        g *= r.nw[21];
        gKy = fmaf(ux * uz, g, gKy);
        gux = fmaf(Kwy * uz, g, gux);
        guz = fmaf(Kwy * ux, g, guz);
        g = Db[1][1][2];
        Db[1][1][2] = r.omw[22] * g;
        g *= r.nw[22];
        gKz = fmaf(ux * uy, g, gKz);
        gux = fmaf(Kwz * uy, g, gux);
        guy = fmaf(Kwz * ux, g, guy);
    }
    // order 4, diagonal: A = xxyy, B = xxzz, C = yyzz
    {
        const float gABn = 0.5f * (Db[2][2][0] + Db[2][0][2]);
        const float g19 = 0.5f * (Db[2][2][0] - Db[2][0][2]);
        const float g17 = third * (2.0f * gABn + Db[0][2][2]);
        const float g18 = third * (gABn - Db[0][2][2]);
        Db[2][2][0] = r.omw[17] * g17 + r.omw[18] * g18 + r.omw[19] * g19;
        Db[2][0][2] = r.omw[17] * g17 + r.omw[18] * g18 - r.omw[19] * g19;
        Db[0][2][2] = r.omw[17] * g17 - 2.0f * r.omw[18] * g18;
        const float gA = r.w[17] * g17 + r.w[18] * g18 + r.w[19] * g19;
        const float gB = r.w[17] * g17 + r.w[18] * g18 - r.w[19] * g19;
        const float gC = r.w[17] * g17 - 2.0f * r.w[18] * g18;
        // dA = Kwx dyy + Kwy dxx + dxx dyy, etc.
        gdx = fmaf(Kwy + dyy, gA, fmaf(Kwz + dzz, gB, gdx));
        gdy = fmaf(Kwx + dxx, gA, fmaf(Kwz + dzz, gC, gdy));
        gdz = fmaf(Kwx + dxx, gB, fmaf(Kwy + dyy, gC, gdz));
        gKx = fmaf(dyy, gA, fmaf(dzz, gB, gKx));
        gKy = fmaf(dxx, gA, fmaf(dzz, gC, gKy));
        gKz = fmaf(dxx, gB, fmaf(dyy, gC, gKz));
    }
    // order 3
    {
        const float gs = 0.5f * (Db[1][2][0] + Db[1][0][2]);
        const float gt = 0.5f * (Db[1][2][0] - Db[1][0][2]);
        const float as = r.w[10] * gs, at = r.w[13] * gt;
        gux = fmaf(as, Kwy + Kwz, fmaf(at, Kwy - Kwz, gux));
        gKy = fmaf(ux, as + at, gKy);
        gKz = fmaf(ux, as - at, gKz);
        const float bs = r.omw[10] * gs, bt = r.omw[13] * gt;
        Db[1][2][0] = bs + bt;
        Db[1][0][2] = bs - bt;
    }
    {
        const float gs = 0.5f * (Db[2][1][0] + Db[0][1][2]);
        const float gt = 0.5f * (Db[2][1][0] - Db[0][1][2]);
        const float as = r.w[11] * gs, at = r.w[14] * gt;
        guy = fmaf(as, Kwx + Kwz, fmaf(at, Kwx - Kwz, guy));
        gKx = fmaf(uy, as + at, gKx);
        gKz = fmaf(uy, as - at, gKz);
        const float bs = r.omw[11] * gs, bt = r.omw[14] * gt;
        Db[2][1][0] = bs + bt;
        Db[0][1][2] = bs - bt;
    }
    {
        const float gs = 0.5f * (Db[2][0][1] + Db[0][2][1]);
        const float gt = 0.5f * (Db[2][0][1] - Db[0][2][1]);
        const float as = r.w[12] * gs, at = r.w[15] * gt;
        guz = fmaf(as, Kwx + Kwy, fmaf(at, Kwx - Kwy, guz));
        gKx = fmaf(uz, as + at, gKx);
        gKy = fmaf(uz, as - at, gKy);
        const float bs = r.omw[12] * gs, bt = r.omw[15] * gt;
        Db[2][0][1] = bs + bt;
        Db[0][2][1] = bs - bt;
    }
    {
        const float g = Db[1][1][1];
        Db[1][1][1] = r.omw[16] * g;
        const float a = r.w[16] * g;
        gux = fmaf(uy * uz, a, gux);
        guy = fmaf(ux * uz, a, guy);
        guz = fmaf(ux * uy, a, guz);
    }
    // order 2, off-diagonal: D~ = omw D + nw u_i u_j
    {
        float g = Db[1][1][0];
        Db[1][1][0] = r.omw[4] * g;
        g *= r.nw[4];
        gux = fmaf(uy, g, gux);
        guy = fmaf(ux, g, guy);
        g = Db[1][0][1];
        Db[1][0][1] = r.omw[5] * g;
        g *= r.nw[5];
        gux = fmaf(uz, g, gux);
        guz = fmaf(ux, g, guz);
        g = Db[0][1][1];
        Db[0][1][1] = r.omw[6] * g;
        g *= r.nw[6];
        guy = fmaf(uz, g, guy);
        guz = fmaf(uy, g, guz);
    }
    // order 2, diagonal (with the adjoints gathered from orders 4 and 6)
    {
        const float ga = 0.5f * (gdx - gdy);
        const float gb = (gdx + gdy) * (1.0f / 6.0f) - gdz * third;
        const float gc = (gdx + gdy + gdz) * third;
        const float a7 = r.nw[7] * ga, a8 = r.nw[8] * gb, a9 = r.w[9] * gc;
        gux = fmaf(2.0f * ux, a7 + a8 - a9, gux);
        guy = fmaf(2.0f * uy, -a7 + a8 - a9, guy);
        guz = fmaf(2.0f * uz, -2.0f * a8 - a9, guz);
        gdrho += a9;
        const float ba = r.omw[7] * ga, bb = r.omw[8] * gb, bc = r.omw[9] * gc;
        Db[2][0][0] = ba + bb + bc;
        Db[0][2][0] = -ba + bb + bc;
        Db[0][0][2] = -2.0f * bb + bc;
    }
    // Kw_i = 1/3 + u_i^2
    gux = fmaf(2.0f * ux, gKx, gux);
    guy = fmaf(2.0f * uy, gKy, guy);
    guz = fmaf(2.0f * uz, gKz, guz);
}

// Adjoint of collide27 for one cell.  f: pre-collision deviations (slot
// order); mu: adjoint of the post-collision values (slot order).  Writes
// lam (slot order) and the force adjoint (gFx, gFy, gFz).
__device__ __forceinline__ void adjoint27(const float (&f)[27], float Fx, float Fy, float Fz,
                                          const Rates27<float> &r, const float (&mu)[27],
                                          float (&lam)[27], float &gFx, float &gFy, float &gFz) {
    // ---- forward recomputation: K (pre-source central moments), Dt
    float K[3][3][3];
    float drho, ux, uy, uz;
    forward27<float>(f, K, Fx, Fy, Fz, drho, ux, uy, uz);
    float Dt[3][3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int p = 0; p < 3; ++p) Dt[m][n][p] = K[m][n][p];
    Dt[1][0][0] += Fx;
    Dt[0][1][0] += Fy;
    Dt[0][0][1] += Fz;
    relax27<float>(Dt, ux, uy, uz, drho, r);

    // ---- reverse of the inverse sweeps: Db = Inv(u)^T mu (x, then y, then z)
    float Db[3][3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float a = mu[s27(0, j, k)], b = mu[s27(1, j, k)], c = mu[s27(2, j, k)];
            inv_line_T(ux, a, b, c);
            Db[0][j][k] = a;
            Db[1][j][k] = b;
            Db[2][j][k] = c;
        }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) inv_line_T(uy, Db[m][0][k], Db[m][1][k], Db[m][2][k]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) inv_line_T(uz, Db[m][n][0], Db[m][n][1], Db[m][n][2]);
    // u through Inv(u): <Db, N Dt>
    float gux, guy, guz;
    shift_u_terms(Db, Dt, gux, guy, guz);
    float gdrho = 0.0f;
    // ---- reverse of the relaxation
    relax27_T(Dt, Db, ux, uy, uz, r, gux, guy, guz, gdrho);
    // ---- source: D = K + sigma(F)
    gFx = Db[1][0][0];
    gFy = Db[0][1][0];
    gFz = Db[0][0][1];
    // ---- u through Shift(u): -<Kbar, N K>
    {
        float sx, sy, sz;
        shift_u_terms(Db, K, sx, sy, sz);
        gux -= sx;
        guy -= sy;
        guz -= sz;
    }
    // ---- reverse of the shifts: Rbar = Shift(u)^T Kbar (z, y, x; they commute)
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) shift_line_T(uz, Db[m][n][0], Db[m][n][1], Db[m][n][2]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int p = 0; p < 3; ++p) shift_line_T(uy, Db[m][0][p], Db[m][1][p], Db[m][2][p]);
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int p = 0; p < 3; ++p) shift_line_T(ux, Db[0][n][p], Db[1][n][p], Db[2][n][p]);
    // ---- u = (j + F/2) / rho
    const float inv_rho = 1.0f / (1.0f + drho);
    const float gjx = gux * inv_rho, gjy = guy * inv_rho, gjz = guz * inv_rho;
    gdrho -= fmaf(ux, gjx, fmaf(uy, gjy, uz * gjz));
    gFx = fmaf(0.5f, gjx, gFx);
    gFy = fmaf(0.5f, gjy, gFy);
    gFz = fmaf(0.5f, gjz, gFz);
    Db[0][0][0] += gdrho;
    Db[1][0][0] += gjx;
    Db[0][1][0] += gjy;
    Db[0][0][1] += gjz;
    // ---- reverse of the raw sums: lam = Sums^T Rbar
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) sums_line_T(Db[m][n][0], Db[m][n][1], Db[m][n][2]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) sums_line_T(Db[m][0][k], Db[m][1][k], Db[m][2][k]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sums_line_T(Db[0][j][k], Db[1][j][k], Db[2][j][k]);
            lam[s27(0, j, k)] = Db[0][j][k];
            lam[s27(1, j, k)] = Db[1][j][k];
            lam[s27(2, j, k)] = Db[2][j][k];
        }
}

}  // namespace lbm
