// Reverse mode of the D3Q15 collision (collide_q15.cuh), written by hand.
//
// The collision maps the pre-collision deviations f and the force F to
//     f~ = f + K.g(s(f), F) + K D^-1 m(F, u),
// with s the signed sums of f over the index sets of App. G (linear in f),
// u = (j + F/2) / rho, g_4..g_14 the cascaded kernels of App. G (each a
// polynomial in s, u, F and the lower kernels) and m the source
// projections.  Given the adjoint mu of f~, adjoint15 returns
// lam = (d f~ / d f)^T mu and Fbar = (d f~ / d F)^T mu:
//   - the update is linear: gbar_beta = <K_beta|mu> and, for the source,
//     mbar_beta = <K_beta|mu> / D_beta (D_beta = <K_beta|K_beta>);
//   - the kernels are reversed from g_14 down to g_4 (the cascade makes the
//     higher kernels depend on the lower ones), accumulating the adjoints of
//     the raw-moment combinations (eta'), of u, rho and F;
//   - those go back through u = (j + F/2) / rho and the sums to lam.
// The source path is always reversed, also where F = 0 (the forward skips
// S there only because it vanishes; its derivative in F does not).
#pragma once

#include "collide_q15.cuh"

namespace lbm {

// <K_beta|K_beta> over the D3Q15 velocities
__host__ __device__ constexpr int d15(int b) {
    int s = 0;
    for (int a = 0; a < 15; ++a) s += k15(b, a) * k15(b, a);
    return s;
}

// Adjoint of collide15 for one cell (V = float) or two (V = f2).  f:
// pre-collision deviations; mu: adjoint of the post-collision values; r:
// the forward's rates (omega_beta / k_beta).  Writes lam and (gFx, gFy, gFz).
template <typename V>
__device__ __forceinline__ void adjoint15(const V (&f)[15], V Fx, V Fy, V Fz,
                                          const Rates15<V> &r, const V (&mu)[15], V (&lam)[15],
                                          V &gFx, V &gFy, V &gFz) {
    const V zero = splat<V>(0.0f), one = splat<V>(1.0f), half = splat<V>(0.5f);
    const V two = splat<V>(2.0f), three = splat<V>(3.0f), eighth = splat<V>(0.125f);
    const V third = splat<V>(1.0f / 3.0f), six = splat<V>(6.0f);

    // ---- forward recomputation (the quantities of kernels15)
    V drho, jx, jy, jz, kxy, kxz, kyz, kxx, kyy, kzz, kxyy, kxxy, kxxz, kxyz, kxxyy;
    sums15(f, drho, jx, jy, jz, kxy, kxz, kyz, kxx, kyy, kzz, kxyy, kxxy, kxxz, kxyz, kxxyy);
    const V rho = one + drho;
    const V inv_rho = vrcp(rho);
    const V ux = vfma(half, Fx, jx) * inv_rho;
    const V uy = vfma(half, Fy, jy) * inv_rho;
    const V uz = vfma(half, Fz, jz) * inv_rho;
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;
    const V fux = Fx * ux, fuy = Fy * uy, fuz = Fz * uz;
    const V exy = kxy + vfma(Fx, uy, Fy * ux);
    const V exz = kxz + vfma(Fx, uz, Fz * ux);
    const V eyz = kyz + vfma(Fy, uz, Fz * uy);
    const V exx = vfma(two, fux, kxx);
    const V eyy = vfma(two, fuy, kyy);
    const V exyy = kxyy + vfma(Fx, uy2, two * fuy * ux);
    const V exxy = kxxy + vfma(Fy, ux2, two * fux * uy);
    const V Exx = third + exx, Eyy = third + eyy;
    // kernels g_4..g_11 (the inputs of the higher ones)
    V g[15];
    g[4] = r.w[4] * (vfma(rho, uxy, half * vfma(Fx, uy, Fy * ux)) - exy);
    g[5] = r.w[5] * (vfma(rho, uxz, half * vfma(Fx, uz, Fz * ux)) - exz);
    g[6] = r.w[6] * (vfma(rho, uyz, half * vfma(Fy, uz, Fz * uy)) - eyz);
    {
        const V ezz = vfma(two, fuz, kzz);
        const V s_u = vfma(Fx, ux, vfma(Fy, uy, Fz * uz));
        g[7] = r.w[7] * (vfma(rho, ux2 - uy2, fux - fuy) - (exx - eyy));
        g[8] = r.w[8] * (vfma(rho, (ux2 + uy2) - two * uz2, (fux + fuy) - two * fuz) -
                         ((exx + eyy) - two * ezz));
        g[9] = r.w[9] * (vfma(rho, ux2 + uy2 + uz2, s_u + drho) - (exx + eyy + ezz));
    }
    g[10] = vfma(r.w[10],
                 vfma(two * uy, exy, ux * Eyy) -
                     vfma(two * rho * ux, uy2, vfma(half * Fx, uy2, Fy * uy * ux)) - exyy,
                 vfma(uy, g[4], eighth * ux * vfma(three, g[9], g[8] - g[7])));
    g[11] = vfma(r.w[11],
                 vfma(two * ux, exy, uy * Exx) -
                     vfma(two * rho * ux2, uy, vfma(half * Fy, ux2, Fx * uxy)) - exxy,
                 vfma(ux, g[4], eighth * uy * vfma(three, g[9], g[8] + g[7])));
    const V dkx = vfma(six, g[9], exx + two * (g[7] + g[8])) - vfma(rho, ux2, fux);
    const V dky = vfma(six, g[9], eyy + two * (g[8] - g[7])) - vfma(rho, uy2, fuy);

    // ---- reverse of the update: projections of mu on the basis
    // On the corners the basis vectors are 1 (K0, K9), 2 (K14), sx, sy, sz
    // (K1..K3, and K10..K12 times 2), sx sy, sx sz, sy sz (K4..K6),
    // sx sy sz (K13), and 0 (K7, K8); on the axis pairs K9 = -1, K14 = -8,
    // K10..K12 = -8 e; at rest K9 = -2, K14 = 32 (k15 above).
    V P[15];
    {
        V Cm, Cx, Cy, Cz, Cxy, Cxz, Cyz, Cxyz, sm, dx, dy, dz, ax, ay, az;
        corner_axis_sums15(mu, Cm, Cx, Cy, Cz, Cxy, Cxz, Cyz, Cxyz, ax, ay, az, dx, dy, dz);
        sm = (ax + ay) + az;
        const V m8 = splat<V>(-8.0f);
        P[0] = (mu[0] + sm) + Cm;
        P[1] = dx + Cx;
        P[2] = dy + Cy;
        P[3] = dz + Cz;
        P[4] = Cxy;
        P[5] = Cxz;
        P[6] = Cyz;
        P[7] = ax - ay;
        P[8] = (ax + ay) - two * az;
        P[9] = vfma(splat<V>(-2.0f), mu[0], Cm - sm);
        P[10] = vfma(m8, dx, two * Cx);
        P[11] = vfma(m8, dy, two * Cy);
        P[12] = vfma(m8, dz, two * Cz);
        P[13] = Cxyz;
        P[14] = vfma(splat<V>(32.0f), mu[0], vfma(m8, sm, two * Cm));
    }
    V bg[15];
#pragma unroll
    for (int b = 4; b < 15; ++b) bg[b] = P[b];

    // adjoint accumulators
    V b_rho = zero, b_drho = zero, b_ux = zero, b_uy = zero, b_uz = zero;
    V b_Fx = zero, b_Fy = zero, b_Fz = zero;
    V b_ux2 = zero, b_uy2 = zero, b_uz2 = zero, b_uxy = zero, b_uxz = zero, b_uyz = zero;
    V b_fux = zero, b_fuy = zero, b_fuz = zero, b_su = zero;
    V b_exy = zero, b_exz = zero, b_eyz = zero, b_exx = zero, b_eyy = zero, b_ezz = zero;
    V b_exyy = zero, b_exxy = zero, b_exxz = zero, b_exyz = zero, b_exxyy = zero;

    // ---- g14 = w14 br14 + B14
    {
        const V bt = bg[14];
        const V b = r.w[14] * bt;
        // B14 = -2 uxy g4 + (ux2 - uy2) g7 / 8 - (ux2 + uy2) g8 / 8
        //       + (-3/8 (ux2 + uy2) - 1/2) g9 + 2 (ux g10 + uy g11)
        const V sxy = ux2 + uy2;
        bg[4] = vfma(splat<V>(-2.0f) * uxy, bt, bg[4]);
        b_uxy = vfma(splat<V>(-2.0f) * g[4], bt, b_uxy);
        bg[7] = vfma(eighth * (ux2 - uy2), bt, bg[7]);
        bg[8] = vfma(splat<V>(-0.125f) * sxy, bt, bg[8]);
        bg[9] = vfma(vfma(splat<V>(-0.375f), sxy, splat<V>(-0.5f)), bt, bg[9]);
        const V c2 = vfma(eighth, g[7] - g[8], splat<V>(-0.375f) * g[9]);  // d B14 / d ux2
        const V c2y = vfma(splat<V>(-0.125f), g[7] + g[8], splat<V>(-0.375f) * g[9]);
        b_ux2 = vfma(c2, bt, b_ux2);
        b_uy2 = vfma(c2y, bt, b_uy2);
        bg[10] = vfma(two * ux, bt, bg[10]);
        bg[11] = vfma(two * uy, bt, bg[11]);
        b_ux = vfma(two * g[10], bt, b_ux);
        b_uy = vfma(two * g[11], bt, b_uy);
        // br14
        b_ux = vfma(two * exyy, b, b_ux);
        b_exyy = vfma(two * ux, b, b_exyy);
        b_uy = vfma(two * exxy, b, b_uy);
        b_exxy = vfma(two * uy, b, b_exxy);
        b_ux2 = b_ux2 - Eyy * b;
        b_eyy = b_eyy - ux2 * b;
        b_uy2 = b_uy2 - Exx * b;
        b_exx = b_exx - uy2 * b;
        b_uxy = vfma(splat<V>(-4.0f) * exy, b, b_uxy);
        b_exy = vfma(splat<V>(-4.0f) * uxy, b, b_exy);
        const V b_dkx = (third + dky) * b;
        const V b_dky = (third + dkx) * b;
        b_rho = vfma(three * ux2 * uy2, b, b_rho);
        b_ux2 = vfma(vfma(three * rho, uy2, Fy * uy), b, b_ux2);
        b_uy2 = vfma(vfma(three * rho, ux2, Fx * ux), b, b_uy2);
        b_Fx = vfma(ux * uy2, b, b_Fx);
        b_Fy = vfma(uy * ux2, b, b_Fy);
        b_ux = vfma(Fx * uy2, b, b_ux);
        b_uy = vfma(Fy * ux2, b, b_uy);
        b_exxyy = b_exxyy - b;
        // dkx = 6 g9 + exx + 2 (g7 + g8) - (rho ux2 + fux)
        bg[9] = vfma(six, b_dkx + b_dky, bg[9]);
        b_exx = b_exx + b_dkx;
        b_eyy = b_eyy + b_dky;
        bg[7] = vfma(two, b_dkx - b_dky, bg[7]);
        bg[8] = vfma(two, b_dkx + b_dky, bg[8]);
        b_rho = b_rho - vfma(ux2, b_dkx, uy2 * b_dky);
        b_ux2 = b_ux2 - rho * b_dkx;
        b_uy2 = b_uy2 - rho * b_dky;
        b_fux = b_fux - b_dkx;
        b_fuy = b_fuy - b_dky;
    }
    // ---- g13 = w13 A13 + uz g4 + uy g5 + ux g6
    {
        const V bt = bg[13];
        const V b = r.w[13] * bt;
        bg[4] = vfma(uz, bt, bg[4]);
        bg[5] = vfma(uy, bt, bg[5]);
        bg[6] = vfma(ux, bt, bg[6]);
        b_uz = vfma(g[4], bt, b_uz);
        b_uy = vfma(g[5], bt, b_uy);
        b_ux = vfma(g[6], bt, b_ux);
        // A13 = ux eyz + uy exz + uz exy - 2 rho ux uyz
        //       - (Fx uyz + Fy uxz + Fz uxy) / 2 - exyz
        b_ux = vfma(eyz - two * rho * uyz, b, b_ux);
        b_eyz = vfma(ux, b, b_eyz);
        b_uy = vfma(exz, b, b_uy);
        b_exz = vfma(uy, b, b_exz);
        b_uz = vfma(exy, b, b_uz);
        b_exy = vfma(uz, b, b_exy);
        b_rho = vfma(splat<V>(-2.0f) * ux * uyz, b, b_rho);
        b_uyz = b_uyz - vfma(two * rho, ux, half * Fx) * b;
        b_uxz = b_uxz - half * Fy * b;
        b_uxy = b_uxy - half * Fz * b;
        b_Fx = b_Fx - half * uyz * b;
        b_Fy = b_Fy - half * uxz * b;
        b_Fz = b_Fz - half * uxy * b;
        b_exyz = b_exyz - b;
    }
    // ---- g12 = w12 A12 + ux g5 + uz (3 g9 + g8 + g7) / 8
    {
        const V bt = bg[12];
        const V b = r.w[12] * bt;
        bg[5] = vfma(ux, bt, bg[5]);
        b_ux = vfma(g[5], bt, b_ux);
        b_uz = vfma(eighth * vfma(three, g[9], g[8] + g[7]), bt, b_uz);
        const V e8 = eighth * uz * bt;
        bg[9] = vfma(three, e8, bg[9]);
        bg[8] = bg[8] + e8;
        bg[7] = bg[7] + e8;
        // A12 = 2 ux exz + uz Exx - 2 rho ux2 uz - Fz ux2 / 2 - Fx uxz - exxz
        b_ux = vfma(two * exz, b, b_ux);
        b_exz = vfma(two * ux, b, b_exz);
        b_uz = vfma(Exx - two * rho * ux2, b, b_uz);
        b_exx = vfma(uz, b, b_exx);
        b_rho = vfma(splat<V>(-2.0f) * ux2 * uz, b, b_rho);
        b_ux2 = b_ux2 - vfma(two * rho, uz, half * Fz) * b;
        b_Fz = b_Fz - half * ux2 * b;
        b_Fx = b_Fx - uxz * b;
        b_uxz = b_uxz - Fx * b;
        b_exxz = b_exxz - b;
    }
    // ---- g11 = w11 A11 + ux g4 + uy (3 g9 + g8 + g7) / 8
    {
        const V bt = bg[11];
        const V b = r.w[11] * bt;
        bg[4] = vfma(ux, bt, bg[4]);
        b_ux = vfma(g[4], bt, b_ux);
        b_uy = vfma(eighth * vfma(three, g[9], g[8] + g[7]), bt, b_uy);
        const V e8 = eighth * uy * bt;
        bg[9] = vfma(three, e8, bg[9]);
        bg[8] = bg[8] + e8;
        bg[7] = bg[7] + e8;
        // A11 = 2 ux exy + uy Exx - 2 rho ux2 uy - Fy ux2 / 2 - Fx uxy - exxy
        b_ux = vfma(two * exy, b, b_ux);
        b_exy = vfma(two * ux, b, b_exy);
        b_uy = vfma(Exx - two * rho * ux2, b, b_uy);
        b_exx = vfma(uy, b, b_exx);
        b_rho = vfma(splat<V>(-2.0f) * ux2 * uy, b, b_rho);
        b_ux2 = b_ux2 - vfma(two * rho, uy, half * Fy) * b;
        b_Fy = b_Fy - half * ux2 * b;
        b_Fx = b_Fx - uxy * b;
        b_uxy = b_uxy - Fx * b;
        b_exxy = b_exxy - b;
    }
    // ---- g10 = w10 A10 + uy g4 + ux (3 g9 + g8 - g7) / 8
    {
        const V bt = bg[10];
        const V b = r.w[10] * bt;
        bg[4] = vfma(uy, bt, bg[4]);
        b_uy = vfma(g[4], bt, b_uy);
        b_ux = vfma(eighth * vfma(three, g[9], g[8] - g[7]), bt, b_ux);
        const V e8 = eighth * ux * bt;
        bg[9] = vfma(three, e8, bg[9]);
        bg[8] = bg[8] + e8;
        bg[7] = bg[7] - e8;
        // A10 = 2 uy exy + ux Eyy - 2 rho ux uy2 - Fx uy2 / 2 - Fy uy ux - exyy
        b_uy = vfma(two * exy - Fy * ux, b, b_uy);
        b_exy = vfma(two * uy, b, b_exy);
        b_ux = vfma(Eyy - vfma(two * rho, uy2, Fy * uy), b, b_ux);
        b_eyy = vfma(ux, b, b_eyy);
        b_rho = vfma(splat<V>(-2.0f) * ux * uy2, b, b_rho);
        b_uy2 = b_uy2 - vfma(two * rho, ux, half * Fx) * b;
        b_Fx = b_Fx - half * uy2 * b;
        b_Fy = b_Fy - uy * ux * b;
        b_exyy = b_exyy - b;
    }
    // ---- g9 = w9 (rho (ux2 + uy2 + uz2) + s_u + drho - (exx + eyy + ezz))
    {
        const V b = r.w[9] * bg[9];
        b_rho = vfma(ux2 + uy2 + uz2, b, b_rho);
        const V rb = rho * b;
        b_ux2 = b_ux2 + rb;
        b_uy2 = b_uy2 + rb;
        b_uz2 = b_uz2 + rb;
        b_su = b_su + b;
        b_drho = b_drho + b;
        b_exx = b_exx - b;
        b_eyy = b_eyy - b;
        b_ezz = b_ezz - b;
    }
    // ---- g8 = w8 (rho (ux2 + uy2 - 2 uz2) + fux + fuy - 2 fuz - (exx + eyy - 2 ezz))
    {
        const V b = r.w[8] * bg[8];
        b_rho = vfma((ux2 + uy2) - two * uz2, b, b_rho);
        const V rb = rho * b;
        b_ux2 = b_ux2 + rb;
        b_uy2 = b_uy2 + rb;
        b_uz2 = b_uz2 - (rb + rb);
        b_fux = b_fux + b;
        b_fuy = b_fuy + b;
        b_fuz = b_fuz - (b + b);
        b_exx = b_exx - b;
        b_eyy = b_eyy - b;
        b_ezz = b_ezz + (b + b);
    }
    // ---- g7 = w7 (rho (ux2 - uy2) + fux - fuy - (exx - eyy))
    {
        const V b = r.w[7] * bg[7];
        b_rho = vfma(ux2 - uy2, b, b_rho);
        const V rb = rho * b;
        b_ux2 = b_ux2 + rb;
        b_uy2 = b_uy2 - rb;
        b_fux = b_fux + b;
        b_fuy = b_fuy - b;
        b_exx = b_exx - b;
        b_eyy = b_eyy + b;
    }
    // ---- g4..g6 = w (rho u_i u_j + (F_i u_j + F_j u_i) / 2 - e_ij)
    {
        const V b = r.w[4] * bg[4];
        b_rho = vfma(uxy, b, b_rho);
        b_uxy = vfma(rho, b, b_uxy);
        b_Fx = vfma(half * uy, b, b_Fx);
        b_uy = vfma(half * Fx, b, b_uy);
        b_Fy = vfma(half * ux, b, b_Fy);
        b_ux = vfma(half * Fy, b, b_ux);
        b_exy = b_exy - b;
    }
    {
        const V b = r.w[5] * bg[5];
        b_rho = vfma(uxz, b, b_rho);
        b_uxz = vfma(rho, b, b_uxz);
        b_Fx = vfma(half * uz, b, b_Fx);
        b_uz = vfma(half * Fx, b, b_uz);
        b_Fz = vfma(half * ux, b, b_Fz);
        b_ux = vfma(half * Fz, b, b_ux);
        b_exz = b_exz - b;
    }
    {
        const V b = r.w[6] * bg[6];
        b_rho = vfma(uyz, b, b_rho);
        b_uyz = vfma(rho, b, b_uyz);
        b_Fy = vfma(half * uz, b, b_Fy);
        b_uz = vfma(half * Fy, b, b_uz);
        b_Fz = vfma(half * uy, b, b_Fz);
        b_uy = vfma(half * Fz, b, b_uy);
        b_eyz = b_eyz - b;
    }
    // ---- source projections: mbar_beta = <K_beta|mu> / D_beta
    {
        const V m1 = P[1] * splat<V>(1.0f / d15(1)), m2 = P[2] * splat<V>(1.0f / d15(2));
        const V m3 = P[3] * splat<V>(1.0f / d15(3)), m4 = P[4] * splat<V>(1.0f / d15(4));
        const V m5 = P[5] * splat<V>(1.0f / d15(5)), m6 = P[6] * splat<V>(1.0f / d15(6));
        const V m7 = P[7] * splat<V>(1.0f / d15(7)), m8 = P[8] * splat<V>(1.0f / d15(8));
        const V m9 = P[9] * splat<V>(1.0f / d15(9)), m10 = P[10] * splat<V>(1.0f / d15(10));
        const V m11 = P[11] * splat<V>(1.0f / d15(11)), m12 = P[12] * splat<V>(1.0f / d15(12));
        const V m13 = P[13] * splat<V>(1.0f / d15(13)), m14 = P[14] * splat<V>(1.0f / d15(14));
        b_Fx = b_Fx + m1;
        b_Fy = b_Fy + m2;
        b_Fz = b_Fz + m3;
        // m4..m6 = F_i u_j + F_j u_i
        b_Fx = vfma(uy, m4, vfma(uz, m5, b_Fx));
        b_Fy = vfma(ux, m4, vfma(uz, m6, b_Fy));
        b_Fz = vfma(ux, m5, vfma(uy, m6, b_Fz));
        b_ux = vfma(Fy, m4, vfma(Fz, m5, b_ux));
        b_uy = vfma(Fx, m4, vfma(Fz, m6, b_uy));
        b_uz = vfma(Fx, m5, vfma(Fy, m6, b_uz));
        // m7 = 2 (fux - fuy), m8 = 2 (fux + fuy - 2 fuz), m9 = 2 (fux + fuy + fuz)
        b_fux = vfma(two, (m7 + m8) + m9, b_fux);
        b_fuy = vfma(two, (m8 - m7) + m9, b_fuy);
        b_fuz = vfma(two, m9 - (m8 + m8), b_fuz);
        // m10 = 5 Fx (3 ux2 + uy2 + uz2) + 10 ux (fuy + fuz) - 13 Fx, and cyclic
        const V five = splat<V>(5.0f), ten = splat<V>(10.0f), m13c = splat<V>(-13.0f);
        b_Fx = vfma(vfma(five, vfma(three, ux2, uy2 + uz2), m13c), m10, b_Fx);
        b_Fy = vfma(vfma(five, vfma(three, uy2, ux2 + uz2), m13c), m11, b_Fy);
        b_Fz = vfma(vfma(five, vfma(three, uz2, ux2 + uy2), m13c), m12, b_Fz);
        const V f5x = five * Fx * m10, f5y = five * Fy * m11, f5z = five * Fz * m12;
        b_ux2 = vfma(three, f5x, b_ux2 + f5y + f5z);
        b_uy2 = vfma(three, f5y, b_uy2 + f5x + f5z);
        b_uz2 = vfma(three, f5z, b_uz2 + f5x + f5y);
        b_ux = vfma(ten * (fuy + fuz), m10, b_ux);
        b_uy = vfma(ten * (fux + fuz), m11, b_uy);
        b_uz = vfma(ten * (fux + fuy), m12, b_uz);
        b_fux = vfma(ten, vfma(uy, m11, uz * m12), b_fux);
        b_fuy = vfma(ten, vfma(ux, m10, uz * m12), b_fuy);
        b_fuz = vfma(ten, vfma(ux, m10, uy * m11), b_fuz);
        // m13 = Fx uyz + Fy uxz + Fz uxy
        b_Fx = vfma(uyz, m13, b_Fx);
        b_Fy = vfma(uxz, m13, b_Fy);
        b_Fz = vfma(uxy, m13, b_Fz);
        b_uyz = vfma(Fx, m13, b_uyz);
        b_uxz = vfma(Fy, m13, b_uxz);
        b_uxy = vfma(Fz, m13, b_uxy);
        // m14 = 20 (fux (3 (uy2 + uz2) - 4) + fuy (3 (ux2 + uz2) - 4)
        //           + fuz (3 (ux2 + uy2) - 4))
        const V t20 = splat<V>(20.0f) * m14, m4c = splat<V>(-4.0f);
        b_fux = vfma(vfma(three, uy2 + uz2, m4c), t20, b_fux);
        b_fuy = vfma(vfma(three, ux2 + uz2, m4c), t20, b_fuy);
        b_fuz = vfma(vfma(three, ux2 + uy2, m4c), t20, b_fuz);
        const V t60 = three * t20;
        b_ux2 = vfma(fuy + fuz, t60, b_ux2);
        b_uy2 = vfma(fux + fuz, t60, b_uy2);
        b_uz2 = vfma(fux + fuy, t60, b_uz2);
    }
    // ---- the raw-moment combinations eta' back to the sums, u and F
    // exy = kxy + Fx uy + Fy ux (and xz, yz)
    b_Fx = vfma(uy, b_exy, vfma(uz, b_exz, b_Fx));
    b_Fy = vfma(ux, b_exy, vfma(uz, b_eyz, b_Fy));
    b_Fz = vfma(ux, b_exz, vfma(uy, b_eyz, b_Fz));
    b_ux = vfma(Fy, b_exy, vfma(Fz, b_exz, b_ux));
    b_uy = vfma(Fx, b_exy, vfma(Fz, b_eyz, b_uy));
    b_uz = vfma(Fx, b_exz, vfma(Fy, b_eyz, b_uz));
    // exx = kxx + 2 fux (and yy, zz)
    b_fux = vfma(two, b_exx, b_fux);
    b_fuy = vfma(two, b_eyy, b_fuy);
    b_fuz = vfma(two, b_ezz, b_fuz);
    // exyy = kxyy + Fx uy2 + 2 fuy ux
    b_Fx = vfma(uy2, b_exyy, b_Fx);
    b_uy2 = vfma(Fx, b_exyy, b_uy2);
    b_fuy = vfma(two * ux, b_exyy, b_fuy);
    b_ux = vfma(two * fuy, b_exyy, b_ux);
    // exxy = kxxy + Fy ux2 + 2 fux uy
    b_Fy = vfma(ux2, b_exxy, b_Fy);
    b_ux2 = vfma(Fy, b_exxy, b_ux2);
    b_fux = vfma(two * uy, b_exxy, b_fux);
    b_uy = vfma(two * fux, b_exxy, b_uy);
    // exxz = kxxz + Fz ux2 + 2 fux uz
    b_Fz = vfma(ux2, b_exxz, b_Fz);
    b_ux2 = vfma(Fz, b_exxz, b_ux2);
    b_fux = vfma(two * uz, b_exxz, b_fux);
    b_uz = vfma(two * fux, b_exxz, b_uz);
    // exyz = kxyz + Fx uyz + Fy uxz + Fz uxy
    b_Fx = vfma(uyz, b_exyz, b_Fx);
    b_Fy = vfma(uxz, b_exyz, b_Fy);
    b_Fz = vfma(uxy, b_exyz, b_Fz);
    b_uyz = vfma(Fx, b_exyz, b_uyz);
    b_uxz = vfma(Fy, b_exyz, b_uxz);
    b_uxy = vfma(Fz, b_exyz, b_uxy);
    // exxyy = kxxyy + 2 (fux uy2 + fuy ux2)
    b_fux = vfma(two * uy2, b_exxyy, b_fux);
    b_uy2 = vfma(two * fux, b_exxyy, b_uy2);
    b_fuy = vfma(two * ux2, b_exxyy, b_fuy);
    b_ux2 = vfma(two * fuy, b_exxyy, b_ux2);
    // s_u = Fx ux + Fy uy + Fz uz, fu_i = F_i u_i
    b_fux = b_fux + b_su;
    b_fuy = b_fuy + b_su;
    b_fuz = b_fuz + b_su;
    b_Fx = vfma(ux, b_fux, b_Fx);
    b_Fy = vfma(uy, b_fuy, b_Fy);
    b_Fz = vfma(uz, b_fuz, b_Fz);
    b_ux = vfma(Fx, b_fux, b_ux);
    b_uy = vfma(Fy, b_fuy, b_uy);
    b_uz = vfma(Fz, b_fuz, b_uz);
    // squares and products of u
    b_ux = vfma(two * ux, b_ux2, vfma(uy, b_uxy, vfma(uz, b_uxz, b_ux)));
    b_uy = vfma(two * uy, b_uy2, vfma(ux, b_uxy, vfma(uz, b_uyz, b_uy)));
    b_uz = vfma(two * uz, b_uz2, vfma(ux, b_uxz, vfma(uy, b_uyz, b_uz)));
    // u = (j + F/2) / rho, rho = 1 + drho
    const V b_jx = b_ux * inv_rho, b_jy = b_uy * inv_rho, b_jz = b_uz * inv_rho;
    gFx = vfma(half, b_jx, b_Fx);
    gFy = vfma(half, b_jy, b_Fy);
    gFz = vfma(half, b_jz, b_Fz);
    b_rho = b_rho - vfma(ux, b_jx, vfma(uy, b_jy, uz * b_jz));
    b_drho = b_drho + b_rho;
    // ---- the sums, transposed: lam = mu + sum_s (d s / d f) sbar
    // each lam_a = mu_a + sum over the sums s of (d s / d f_a) sbar: on the
    // corners a sign pattern of 8 coefficients (a butterfly, as in update15)
    {
        const V ex = b_drho + b_exx, ey = b_drho + b_eyy, ez = b_drho + b_ezz;
        lam[0] = mu[0] + b_drho;
        static_for<6>([&](auto ia) {
            constexpr int a = 1 + decltype(ia)::value;
            constexpr int x = q15_e(a, 0), y = q15_e(a, 1), z = q15_e(a, 2);
            V v;
            if constexpr (x > 0) v = ex + b_jx;
            if constexpr (x < 0) v = ex - b_jx;
            if constexpr (y > 0) v = ey + b_jy;
            if constexpr (y < 0) v = ey - b_jy;
            if constexpr (z > 0) v = ez + b_jz;
            if constexpr (z < 0) v = ez - b_jz;
            lam[a] = mu[a] + v;
        });
        const V c0 = ((ex + b_eyy) + (b_ezz + b_exxyy));
        const V cx = b_jx + b_exyy, cy = b_jy + b_exxy, cz = b_jz + b_exxz;
        V A[2], Bx[2], By[2], Bxy[2];
        A[0] = c0 + cz;
        A[1] = c0 - cz;
        Bx[0] = cx + b_exz;
        Bx[1] = cx - b_exz;
        By[0] = cy + b_eyz;
        By[1] = cy - b_eyz;
        Bxy[0] = b_exy + b_exyz;
        Bxy[1] = b_exy - b_exyz;
        static_for<8>([&](auto ic) {
            constexpr int a = 7 + decltype(ic)::value;
            constexpr int x = q15_e(a, 0), y = q15_e(a, 1), z = q15_e(a, 2);
            constexpr int k = z > 0 ? 0 : 1;
            const V P2 = y > 0 ? A[k] + By[k] : A[k] - By[k];
            const V R2 = y > 0 ? Bx[k] + Bxy[k] : Bx[k] - Bxy[k];
            lam[a] = mu[a] + (x > 0 ? P2 + R2 : P2 - R2);
        });
    }
}

}  // namespace lbm
