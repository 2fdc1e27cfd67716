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
//
// Templated on the value type like the forward collision: V = float for one
// cell, V = f2 for two neighbouring cells in packed f32x2 arithmetic (no
// negation of a packed variable: differences are written as subtractions or
// as products with negative constants).
#pragma once

#include "collide_q27.cuh"

namespace lbm {

// transpose of dist_from_central: (abar, bbar, cbar) -> (k0bar, k1bar, k2bar)
template <typename V>
__device__ __forceinline__ void inv_line_T(V u, V u2, V &a, V &b, V &c) {
    const V half = splat<V>(0.5f);
    const V P = half * (a + c) - b;
    const V s = half * (c - a);
    const V k1 = vfma(u2, P, s);             // 2u P + s
    const V k0 = vfma(u, vfma(u, P, s), b);  // b + u s + u^2 P
    a = k0;
    b = k1;
    c = P;
}

// transpose of central_from_sums: (k0bar, k1bar, k2bar) -> (s0bar, s1bar, s2bar);
// nu = -u, nu2 = -2u
template <typename V>
__device__ __forceinline__ void shift_line_T(V nu, V nu2, V &k0, V &k1, V &k2) {
    const V s0 = vfma(nu, vfma(nu, k2, k1), k0);  // k0 - u k1 + u^2 k2
    const V s1 = vfma(nu2, k2, k1);               // k1 - 2u k2
    k0 = s0;
    k1 = s1;
}

// transpose of sums: (s0bar, s1bar, s2bar) -> (abar, bbar, cbar)
template <typename V>
__device__ __forceinline__ void sums_line_T(V &s0, V &s1, V &s2) {
    const V t = s0 + s2;
    const V a = t - s1;
    const V c = t + s1;
    s2 = c;
    s1 = s0;
    s0 = a;
}

// <Dbar, N_x D> etc.: sum over lines of Dbar[1] D[0] + 2 Dbar[2] D[1]
template <typename V>
__device__ __forceinline__ void shift_u_terms(const V (&Db)[3][3][3], const V (&D)[3][3][3],
                                              V &gx, V &gy, V &gz) {
    const V zero = splat<V>(0.0f), two = splat<V>(2.0f);
    V x1 = zero, x2 = zero, y1 = zero, y2 = zero, z1 = zero, z2 = zero;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            x1 = vfma(Db[1][a][b], D[0][a][b], x1);
            x2 = vfma(Db[2][a][b], D[1][a][b], x2);
            y1 = vfma(Db[a][1][b], D[a][0][b], y1);
            y2 = vfma(Db[a][2][b], D[a][1][b], y2);
            z1 = vfma(Db[a][b][1], D[a][b][0], z1);
            z2 = vfma(Db[a][b][2], D[a][b][1], z2);
        }
    gx = vfma(two, x2, x1);
    gy = vfma(two, y2, y1);
    gz = vfma(two, z2, z1);
}

// Reverse of relax27.  Dt: post-collision moments (forward output); Db: on
// input the adjoint of Dt, on output the adjoint of the pre-relaxation D.
// Accumulates the adjoints of u and drho.
template <typename V>
__device__ __forceinline__ void relax27_T(const V (&Dt)[3][3][3], V (&Db)[3][3][3], V ux, V uy,
                                          V uz, const Rates27<V> &r, V &gux, V &guy, V &guz,
                                          V &gdrho) {
    const V third = splat<V>(1.0f / 3.0f), sixth = splat<V>(1.0f / 6.0f);
    const V nthird = splat<V>(-1.0f / 3.0f);
    const V half = splat<V>(0.5f), two = splat<V>(2.0f), zero = splat<V>(0.0f);
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V Kwx = third + ux2, Kwy = third + uy2, Kwz = third + uz2;
    const V dxx = Dt[2][0][0], dyy = Dt[0][2][0], dzz = Dt[0][0][2];
    V gKx = zero, gKy = zero, gKz = zero;                 // adjoints of Kw_i
    V gdx = Db[2][0][0], gdy = Db[0][2][0], gdz = Db[0][0][2];  // of dxx, dyy, dzz

    // order 6: dK = kt_x kt_y kt_z - Kw_x Kw_y Kw_z
    {
        const V ktx = Kwx + dxx, kty = Kwy + dyy, ktz = Kwz + dzz;
        const V g = Db[2][2][2];
        Db[2][2][2] = r.omw[26] * g;
        const V gK = r.w[26] * g;
        gdx = vfma(kty * ktz, gK, gdx);
        gdy = vfma(ktx * ktz, gK, gdy);
        gdz = vfma(ktx * kty, gK, gdz);
        // kt_y kt_z - Kw_y Kw_z etc., in the cancellation-free form
        gKx = vfma(vfma(Kwy, dzz, vfma(Kwz, dyy, dyy * dzz)), gK, gKx);
        gKy = vfma(vfma(Kwx, dzz, vfma(Kwz, dxx, dxx * dzz)), gK, gKy);
        gKz = vfma(vfma(Kwx, dyy, vfma(Kwy, dxx, dxx * dyy)), gK, gKz);
    }
    // order 5
    {
        V g = Db[1][2][2];
        Db[1][2][2] = r.omw[23] * g;
        g = r.w[23] * g;
        gux = vfma(Kwy * Kwz, g, gux);
        gKy = vfma(ux * Kwz, g, gKy);
        gKz = vfma(ux * Kwy, g, gKz);
        g = Db[2][1][2];
        Db[2][1][2] = r.omw[24] * g;
        g = r.w[24] * g;
        guy = vfma(Kwx * Kwz, g, guy);
        gKx = vfma(uy * Kwz, g, gKx);
        gKz = vfma(uy * Kwx, g, gKz);
        g = Db[2][2][1];
        Db[2][2][1] = r.omw[25] * g;
        g = r.w[25] * g;
        guz = vfma(Kwx * Kwy, g, guz);
        gKx = vfma(uz * Kwy, g, gKx);
        gKy = vfma(uz * Kwx, g, gKy);
    }
    // order 4, mixed: D~ = omw D + nw Kw_i u_j u_k
    {
        V g = Db[2][1][1];
        Db[2][1][1] = r.omw[20] * g;
        g = r.nw[20] * g;
        gKx = vfma(uy * uz, g, gKx);
        guy = vfma(Kwx * uz, g, guy);
        guz = vfma(Kwx * uy, g, guz);
        g = Db[1][2][1];
        Db[1][2][1] = r.omw[21] * g;
        g = r.nw[21] * g;
        gKy = vfma(ux * uz, g, gKy);
        gux = vfma(Kwy * uz, g, gux);
        guz = vfma(Kwy * ux, g, guz);
        g = Db[1][1][2];
        Db[1][1][2] = r.omw[22] * g;
        g = r.nw[22] * g;
        gKz = vfma(ux * uy, g, gKz);
        gux = vfma(Kwz * uy, g, gux);
        guy = vfma(Kwz * ux, g, guy);
    }
    // order 4, diagonal: A = xxyy, B = xxzz, C = yyzz
    {
        const V gABn = half * (Db[2][2][0] + Db[2][0][2]);
        const V g19 = half * (Db[2][2][0] - Db[2][0][2]);
        const V g17 = third * vfma(two, gABn, Db[0][2][2]);
        const V g18 = third * (gABn - Db[0][2][2]);
        {
            const V a17 = r.omw[17] * g17, a18 = r.omw[18] * g18, a19 = r.omw[19] * g19;
            const V t = a17 + a18;
            Db[2][2][0] = t + a19;
            Db[2][0][2] = t - a19;
            Db[0][2][2] = a17 - (a18 + a18);
        }
        const V b17 = r.w[17] * g17, b18 = r.w[18] * g18, b19 = r.w[19] * g19;
        const V t = b17 + b18;
        const V gA = t + b19;
        const V gB = t - b19;
        const V gC = b17 - (b18 + b18);
        // dA = Kwx dyy + Kwy dxx + dxx dyy, etc.
        const V kx = Kwx + dxx, ky = Kwy + dyy, kz = Kwz + dzz;
        gdx = vfma(ky, gA, vfma(kz, gB, gdx));
        gdy = vfma(kx, gA, vfma(kz, gC, gdy));
        gdz = vfma(kx, gB, vfma(ky, gC, gdz));
        gKx = vfma(dyy, gA, vfma(dzz, gB, gKx));
        gKy = vfma(dxx, gA, vfma(dzz, gC, gKy));
        gKz = vfma(dxx, gB, vfma(dyy, gC, gKz));
    }
    // order 3
    {
        const V gs = half * (Db[1][2][0] + Db[1][0][2]);
        const V gt = half * (Db[1][2][0] - Db[1][0][2]);
        const V as = r.w[10] * gs, at = r.w[13] * gt;
        gux = vfma(as, Kwy + Kwz, vfma(at, Kwy - Kwz, gux));
        gKy = vfma(ux, as + at, gKy);
        gKz = vfma(ux, as - at, gKz);
        const V bs = r.omw[10] * gs, bt = r.omw[13] * gt;
        Db[1][2][0] = bs + bt;
        Db[1][0][2] = bs - bt;
    }
    {
        const V gs = half * (Db[2][1][0] + Db[0][1][2]);
        const V gt = half * (Db[2][1][0] - Db[0][1][2]);
        const V as = r.w[11] * gs, at = r.w[14] * gt;
        guy = vfma(as, Kwx + Kwz, vfma(at, Kwx - Kwz, guy));
        gKx = vfma(uy, as + at, gKx);
        gKz = vfma(uy, as - at, gKz);
        const V bs = r.omw[11] * gs, bt = r.omw[14] * gt;
        Db[2][1][0] = bs + bt;
        Db[0][1][2] = bs - bt;
    }
    {
        const V gs = half * (Db[2][0][1] + Db[0][2][1]);
        const V gt = half * (Db[2][0][1] - Db[0][2][1]);
        const V as = r.w[12] * gs, at = r.w[15] * gt;
        guz = vfma(as, Kwx + Kwy, vfma(at, Kwx - Kwy, guz));
        gKx = vfma(uz, as + at, gKx);
        gKy = vfma(uz, as - at, gKy);
        const V bs = r.omw[12] * gs, bt = r.omw[15] * gt;
        Db[2][0][1] = bs + bt;
        Db[0][2][1] = bs - bt;
    }
    {
        const V g = Db[1][1][1];
        Db[1][1][1] = r.omw[16] * g;
        const V a = r.w[16] * g;
        gux = vfma(uy * uz, a, gux);
        guy = vfma(ux * uz, a, guy);
        guz = vfma(ux * uy, a, guz);
    }
    // order 2, off-diagonal: D~ = omw D + nw u_i u_j
    {
        V g = Db[1][1][0];
        Db[1][1][0] = r.omw[4] * g;
        g = r.nw[4] * g;
        gux = vfma(uy, g, gux);
        guy = vfma(ux, g, guy);
        g = Db[1][0][1];
        Db[1][0][1] = r.omw[5] * g;
        g = r.nw[5] * g;
        gux = vfma(uz, g, gux);
        guz = vfma(ux, g, guz);
        g = Db[0][1][1];
        Db[0][1][1] = r.omw[6] * g;
        g = r.nw[6] * g;
        guy = vfma(uz, g, guy);
        guz = vfma(uy, g, guz);
    }
    // order 2, diagonal (with the adjoints gathered from orders 4 and 6)
    {
        const V sxy = gdx + gdy;
        const V ga = half * (gdx - gdy);
        const V gb = vfma(nthird, gdz, sixth * sxy);
        const V gc = third * (sxy + gdz);
        const V a7 = r.nw[7] * ga, a8 = r.nw[8] * gb, a9 = r.w[9] * gc;
        gux = vfma(ux + ux, (a7 + a8) - a9, gux);
        guy = vfma(uy + uy, (a8 - a7) - a9, guy);
        guz = guz - (uz + uz) * ((a8 + a8) + a9);
        gdrho = gdrho + a9;
        const V ba = r.omw[7] * ga, bb = r.omw[8] * gb, bc = r.omw[9] * gc;
        const V t = bb + bc;
        Db[2][0][0] = t + ba;
        Db[0][2][0] = t - ba;
        Db[0][0][2] = bc - (bb + bb);
    }
    // Kw_i = 1/3 + u_i^2
    gux = vfma(ux + ux, gKx, gux);
    guy = vfma(uy + uy, gKy, guy);
    guz = vfma(uz + uz, gKz, guz);
}

// Adjoint of collide27 for one cell (V = float) or two (V = f2).  f:
// pre-collision deviations (slot order); mu: adjoint of the post-collision
// values (slot order).  Writes lam (slot order) and the force adjoint
// (gFx, gFy, gFz).
template <typename V>
__device__ __forceinline__ void adjoint27(const V (&f)[27], V Fx, V Fy, V Fz,
                                          const Rates27<V> &r, const V (&mu)[27], V (&lam)[27],
                                          V &gFx, V &gFy, V &gFz) {
    const V zero = splat<V>(0.0f), half = splat<V>(0.5f);
    // ---- forward recomputation: K (pre-source central moments), Dt
    V K[3][3][3];
    V drho, ux, uy, uz;
    forward27<V>(f, K, Fx, Fy, Fz, drho, ux, uy, uz);
    V Dt[3][3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int p = 0; p < 3; ++p) Dt[m][n][p] = K[m][n][p];
    Dt[1][0][0] = Dt[1][0][0] + Fx;
    Dt[0][1][0] = Dt[0][1][0] + Fy;
    Dt[0][0][1] = Dt[0][0][1] + Fz;
    relax27<V>(Dt, ux, uy, uz, drho, r);

    // ---- reverse of the inverse sweeps: Db = Inv(u)^T mu (x, then y, then z)
    V Db[3][3][3];
    {
        const V ux2 = ux + ux, uy2 = uy + uy, uz2 = uz + uz;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                V a = mu[s27(0, j, k)], b = mu[s27(1, j, k)], c = mu[s27(2, j, k)];
                inv_line_T(ux, ux2, a, b, c);
                Db[0][j][k] = a;
                Db[1][j][k] = b;
                Db[2][j][k] = c;
            }
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int k = 0; k < 3; ++k) inv_line_T(uy, uy2, Db[m][0][k], Db[m][1][k], Db[m][2][k]);
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int n = 0; n < 3; ++n) inv_line_T(uz, uz2, Db[m][n][0], Db[m][n][1], Db[m][n][2]);
    }
    // u through Inv(u): <Db, N Dt>
    V gux, guy, guz;
    shift_u_terms(Db, Dt, gux, guy, guz);
    V gdrho = zero;
    // ---- reverse of the relaxation
    relax27_T(Dt, Db, ux, uy, uz, r, gux, guy, guz, gdrho);
    // ---- source: D = K + sigma(F)
    gFx = Db[1][0][0];
    gFy = Db[0][1][0];
    gFz = Db[0][0][1];
    // ---- u through Shift(u): -<Kbar, N K>
    {
        V sx, sy, sz;
        shift_u_terms(Db, K, sx, sy, sz);
        gux = gux - sx;
        guy = guy - sy;
        guz = guz - sz;
    }
    // ---- reverse of the shifts: Rbar = Shift(u)^T Kbar (z, y, x; they commute)
    {
        const V nux = zero - ux, nuy = zero - uy, nuz = zero - uz;
        const V nux2 = nux + nux, nuy2 = nuy + nuy, nuz2 = nuz + nuz;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int n = 0; n < 3; ++n)
                shift_line_T(nuz, nuz2, Db[m][n][0], Db[m][n][1], Db[m][n][2]);
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int p = 0; p < 3; ++p)
                shift_line_T(nuy, nuy2, Db[m][0][p], Db[m][1][p], Db[m][2][p]);
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int p = 0; p < 3; ++p)
                shift_line_T(nux, nux2, Db[0][n][p], Db[1][n][p], Db[2][n][p]);
    }
    // ---- u = (j + F/2) / rho
    const V inv_rho = vrcp(splat<V>(1.0f) + drho);
    const V gjx = gux * inv_rho, gjy = guy * inv_rho, gjz = guz * inv_rho;
    gdrho = gdrho - vfma(ux, gjx, vfma(uy, gjy, uz * gjz));
    gFx = vfma(half, gjx, gFx);
    gFy = vfma(half, gjy, gFy);
    gFz = vfma(half, gjz, gFz);
    Db[0][0][0] = Db[0][0][0] + gdrho;
    Db[1][0][0] = Db[1][0][0] + gjx;
    Db[0][1][0] = Db[0][1][0] + gjy;
    Db[0][0][1] = Db[0][0][1] + gjz;
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
