// D3Q27 central-moment collision with forcing, in registers, on deviations.
//
// The collision of Sec. 7 relaxes, in cascade order, the central moments
// P_beta of the pre-collision state toward the factorised attractors of
// Eq. transformedcentralmomentattractors:
//   order 2:  xy, xz, yz (omega_4..6); xx-yy, xx+yy-2zz, xx+yy+zz (omega_7..9)
//   order 3:  xyy+xzz, xxy+yzz, xxz+yyz, xyy-xzz, xxy-yzz, xxz-yyz, xyz
//             (omega_10..16)
//   order 4:  xxyy+xxzz+yyzz, xxyy+xxzz-2yyzz, xxyy-xxzz, xxyz, xyyz, xyzz
//             (omega_17..22)
//   order 5:  xyyzz, xxyzz, xxyyz (omega_23..25);  order 6: xxyyzz (omega_26)
// each post-collision value being c + omega_beta (c^at - c); density and the
// first central moments are invariant.  Because the cascade's coupling
// matrix <P_beta(e - u)|K_gamma> is lower triangular, this equals
// f~ = f + K.g + S of Eq. cascadedcollision1 with the g of Sec. 7.
//
// GB300 design (not the paper's raw-moment expansion): the D3Q27 monomials
// e_x^m e_y^n e_z^p, m, n, p <= 2, form a tensor product of three 1-D
// three-point spaces, so the central moments about u are three sweeps of
// nine 1-D shifts (x, then y, then z) and the way back is the same sweeps
// reversed -- about 400 FLOP in registers instead of the 27 x 27 products.
// The source enters as its central moments: on D3Q27 they are (0, F, 0, ...)
// (Eq. discretecentralsources), so S is never formed in velocity space.
//
// Precision: every quantity is a deviation from the rest state w_alpha
// (rho = 1, u = 0).  The central moments of w about u factorise into
// k0 = 1, k1 = -u_i, k2 = 1/3 + u_i^2 per axis, so they are known in closed
// form and subtracted analytically; the relaxation is written for
// d = kappa - kappa^w, which keeps O(1) terms out of every FP32 rounding.
#pragma once

#include "lattice.cuh"

namespace lbm {

// slot (paper order) of the D3Q27 velocity with components (i-1, j-1, k-1)
__host__ __device__ constexpr int s27(int i, int j, int k) { return slot_of<27>(i - 1, j - 1, k - 1); }

struct RelaxRates27 {
    float w[27];  // omega_beta; 0..3 unused
};

// 1-D shift of the triple (f(-1), f(0), f(+1)) to central moments about u.
// In: raw sums already formed (s0 = a + b + c, s1 = c - a, s2 = a + c).
__device__ __forceinline__ void central_from_sums(float u, float &m0, float &m1, float &m2) {
    // m0 = s0; m1 = s1 - u s0; m2 = s2 - 2 u s1 + u^2 s0 = s2 - u (s1 + m1)
    const float k1 = fmaf(-u, m0, m1);
    const float k2 = fmaf(-u, m1 + k1, m2);
    m1 = k1;
    m2 = k2;
}

__device__ __forceinline__ void sums(float a, float b, float c, float &s0, float &s1, float &s2) {
    const float ac = a + c;
    s0 = ac + b;
    s1 = c - a;
    s2 = ac;
}

// Inverse: central moments (k0, k1, k2) about u -> (f(-1), f(0), f(+1)).
__device__ __forceinline__ void dist_from_central(float u, float k0, float k1, float k2, float &a,
                                                  float &b, float &c) {
    const float m1 = fmaf(u, k0, k1);      // raw first moment
    const float m2 = fmaf(u, k1 + m1, k2); // raw second moment
    b = k0 - m2;
    c = 0.5f * (m2 + m1);
    a = 0.5f * (m2 - m1);
}

// Relax the deviation central moments D[m][n][p] (= kappa - kappa^w,
// source included) in place.  drho = rho - 1.
__device__ __forceinline__ void relax27(float (&D)[3][3][3], float ux, float uy, float uz,
                                        float drho, const RelaxRates27 &r) {
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const float third = 1.0f / 3.0f;
    const float Kwx = third + ux2, Kwy = third + uy2, Kwz = third + uz2;

    // order 2, off-diagonal: attractor 0, kappa^w = u_i u_j
    D[1][1][0] = fmaf(1.0f - r.w[4], D[1][1][0], -r.w[4] * ux * uy);
    D[1][0][1] = fmaf(1.0f - r.w[5], D[1][0][1], -r.w[5] * ux * uz);
    D[0][1][1] = fmaf(1.0f - r.w[6], D[0][1][1], -r.w[6] * uy * uz);

    // order 2, diagonal: xx-yy -> 0, xx+yy-2zz -> 0, xx+yy+zz -> rho
    {
        float a = D[2][0][0] - D[0][2][0];
        float b = D[2][0][0] + D[0][2][0] - 2.0f * D[0][0][2];
        float c = D[2][0][0] + D[0][2][0] + D[0][0][2];
        a = fmaf(1.0f - r.w[7], a, -r.w[7] * (ux2 - uy2));
        b = fmaf(1.0f - r.w[8], b, -r.w[8] * (ux2 + uy2 - 2.0f * uz2));
        c = fmaf(1.0f - r.w[9], c, r.w[9] * (drho - (ux2 + uy2 + uz2)));
        const float c3 = c * third, b6 = b * (1.0f / 6.0f);
        D[2][0][0] = c3 + b6 + 0.5f * a;
        D[0][2][0] = c3 + b6 - 0.5f * a;
        D[0][0][2] = c3 - 2.0f * b6;
    }
    const float dxx = D[2][0][0], dyy = D[0][2][0], dzz = D[0][0][2];  // post-collision

    // order 3: attractors 0; kappa^w_xyy = -u_x Kw_y etc.
    {
        float s = D[1][2][0] + D[1][0][2], t = D[1][2][0] - D[1][0][2];
        s = fmaf(1.0f - r.w[10], s, r.w[10] * ux * (Kwy + Kwz));
        t = fmaf(1.0f - r.w[13], t, r.w[13] * ux * (Kwy - Kwz));
        D[1][2][0] = 0.5f * (s + t);
        D[1][0][2] = 0.5f * (s - t);
    }
    {
        float s = D[2][1][0] + D[0][1][2], t = D[2][1][0] - D[0][1][2];
        s = fmaf(1.0f - r.w[11], s, r.w[11] * uy * (Kwx + Kwz));
        t = fmaf(1.0f - r.w[14], t, r.w[14] * uy * (Kwx - Kwz));
        D[2][1][0] = 0.5f * (s + t);
        D[0][1][2] = 0.5f * (s - t);
    }
    {
        float s = D[2][0][1] + D[0][2][1], t = D[2][0][1] - D[0][2][1];
        s = fmaf(1.0f - r.w[12], s, r.w[12] * uz * (Kwx + Kwy));
        t = fmaf(1.0f - r.w[15], t, r.w[15] * uz * (Kwx - Kwy));
        D[2][0][1] = 0.5f * (s + t);
        D[0][2][1] = 0.5f * (s - t);
    }
    D[1][1][1] = fmaf(1.0f - r.w[16], D[1][1][1], r.w[16] * ux * uy * uz);

    // order 4: xxyy, xxzz, yyzz -> products of the post-collision kappa~_ii
    {
        const float dA = fmaf(Kwx, dyy, fmaf(Kwy, dxx, dxx * dyy));  // kt_x kt_y - Kw_x Kw_y
        const float dB = fmaf(Kwx, dzz, fmaf(Kwz, dxx, dxx * dzz));
        const float dC = fmaf(Kwy, dzz, fmaf(Kwz, dyy, dyy * dzz));
        const float A = D[2][2][0], B = D[2][0][2], C = D[0][2][2];
        float p17 = A + B + C, p18 = A + B - 2.0f * C, p19 = A - B;
        p17 = fmaf(1.0f - r.w[17], p17, r.w[17] * (dA + dB + dC));
        p18 = fmaf(1.0f - r.w[18], p18, r.w[18] * (dA + dB - 2.0f * dC));
        p19 = fmaf(1.0f - r.w[19], p19, r.w[19] * (dA - dB));
        const float Cn = (p17 - p18) * third;
        const float ABn = (2.0f * p17 + p18) * third;
        D[2][2][0] = 0.5f * (ABn + p19);
        D[2][0][2] = 0.5f * (ABn - p19);
        D[0][2][2] = Cn;
    }
    // xxyz, xyyz, xyzz -> 0; kappa^w_xxyz = Kw_x u_y u_z etc.
    D[2][1][1] = fmaf(1.0f - r.w[20], D[2][1][1], -r.w[20] * Kwx * uy * uz);
    D[1][2][1] = fmaf(1.0f - r.w[21], D[1][2][1], -r.w[21] * ux * Kwy * uz);
    D[1][1][2] = fmaf(1.0f - r.w[22], D[1][1][2], -r.w[22] * ux * uy * Kwz);

    // order 5 -> 0; kappa^w_xyyzz = -u_x Kw_y Kw_z etc.
    D[1][2][2] = fmaf(1.0f - r.w[23], D[1][2][2], r.w[23] * ux * Kwy * Kwz);
    D[2][1][2] = fmaf(1.0f - r.w[24], D[2][1][2], r.w[24] * uy * Kwx * Kwz);
    D[2][2][1] = fmaf(1.0f - r.w[25], D[2][2][1], r.w[25] * uz * Kwx * Kwy);

    // order 6: xxyyzz -> kt_x kt_y kt_z
    {
        const float dK = dxx * Kwy * Kwz + dyy * Kwx * Kwz + dzz * Kwx * Kwy +
                         dxx * dyy * Kwz + dxx * dzz * Kwy + dyy * dzz * Kwx + dxx * dyy * dzz;
        D[2][2][2] = fmaf(1.0f - r.w[26], D[2][2][2], r.w[26] * dK);
    }
}

// Forward transform of deviations f[slot] into raw-sum / central-moment
// space.  Returns drho, j and u; D holds the central moments about u of the
// deviations, to which the caller adds the source.
__device__ __forceinline__ void forward27(const float (&f)[27], float (&D)[3][3][3], float Fx,
                                          float Fy, float Fz, float &drho, float &ux, float &uy,
                                          float &uz) {
    // x: raw sums of each (y, z) line
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            sums(f[s27(0, j, k)], f[s27(1, j, k)], f[s27(2, j, k)], D[0][j][k], D[1][j][k],
                 D[2][j][k]);
    // y: raw sums over y of each x-moment line
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float s0, s1, s2;
            sums(D[m][0][k], D[m][1][k], D[m][2][k], s0, s1, s2);
            D[m][0][k] = s0;
            D[m][1][k] = s1;
            D[m][2][k] = s2;
        }
    // z
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            float s0, s1, s2;
            sums(D[m][n][0], D[m][n][1], D[m][n][2], s0, s1, s2);
            D[m][n][0] = s0;
            D[m][n][1] = s1;
            D[m][n][2] = s2;
        }
    // D now holds raw moments of the deviations; the rest state has raw
    // moments (1, 0, 1/3, ...) which sum to rho = 1 + drho, j = j_dev.
    drho = D[0][0][0];
    const float inv_rho = 1.0f / (1.0f + drho);
    ux = (D[1][0][0] + 0.5f * Fx) * inv_rho;
    uy = (D[0][1][0] + 0.5f * Fy) * inv_rho;
    uz = (D[0][0][1] + 0.5f * Fz) * inv_rho;
    // shift raw -> central about u, one axis at a time (the shifts commute)
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int p = 0; p < 3; ++p) central_from_sums(ux, D[0][n][p], D[1][n][p], D[2][n][p]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int p = 0; p < 3; ++p) central_from_sums(uy, D[m][0][p], D[m][1][p], D[m][2][p]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) central_from_sums(uz, D[m][n][0], D[m][n][1], D[m][n][2]);
}

// Inverse transform: deviation central moments about u -> deviations f[slot].
__device__ __forceinline__ void inverse27(float (&D)[3][3][3], float ux, float uy, float uz,
                                          float (&f)[27]) {
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            float a, b, c;
            dist_from_central(uz, D[m][n][0], D[m][n][1], D[m][n][2], a, b, c);
            D[m][n][0] = a;
            D[m][n][1] = b;
            D[m][n][2] = c;
        }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float a, b, c;
            dist_from_central(uy, D[m][0][k], D[m][1][k], D[m][2][k], a, b, c);
            D[m][0][k] = a;
            D[m][1][k] = b;
            D[m][2][k] = c;
        }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dist_from_central(ux, D[0][j][k], D[1][j][k], D[2][j][k], f[s27(0, j, k)],
                              f[s27(1, j, k)], f[s27(2, j, k)]);
}

// One cell: pre-collision deviations in, post-collision deviations out
// (both f - w, slot order).  (Fx, Fy, Fz): the cell's body force.
__device__ __forceinline__ void collide27(float (&f)[27], float Fx, float Fy, float Fz,
                                          const RelaxRates27 &r) {
    float D[3][3][3];
    float drho, ux, uy, uz;
    forward27(f, D, Fx, Fy, Fz, drho, ux, uy, uz);
    // central moments of the source: F at first order (Eq. discretecentralsources)
    D[1][0][0] += Fx;
    D[0][1][0] += Fy;
    D[0][0][1] += Fz;
    // d = kappa - kappa^w: the rest state's central moments about u are
    // k_m(u_x) k_n(u_y) k_p(u_z), with deviations counted from them.  The
    // forward sweep produced central moments of the deviations, i.e. d
    // already (kappa^w is the part carried by w itself).
    relax27(D, ux, uy, uz, drho, r);
    inverse27(D, ux, uy, uz, f);
}

// Deviations of the initial state f = f^at(rho, u) - S/2 at one cell
// (the post-collision state of a collision with every omega = 1 and no force,
// shifted by half the source, whose central moments are (0, F, 0, ...)).
__device__ __forceinline__ void equilibrium27(float drho, float ux, float uy, float uz, float Fx,
                                              float Fy, float Fz, float (&f)[27]) {
    const float third = 1.0f / 3.0f;
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const float Kwx = third + ux2, Kwy = third + uy2, Kwz = third + uz2;
    float D[3][3][3];
    // central moments of f^at minus those of w (k0 = 1, k1 = -u, k2 = Kw)
    D[0][0][0] = drho;
    D[1][0][0] = ux - 0.5f * Fx;  // first central moment of f^at - S/2 is -F/2
    D[0][1][0] = uy - 0.5f * Fy;
    D[0][0][1] = uz - 0.5f * Fz;
    D[1][1][0] = -ux * uy;
    D[1][0][1] = -ux * uz;
    D[0][1][1] = -uy * uz;
    const float dii = drho * third;  // rho/3 - 1/3
    D[2][0][0] = dii - ux2;
    D[0][2][0] = dii - uy2;
    D[0][0][2] = dii - uz2;
    D[1][2][0] = ux * Kwy;
    D[1][0][2] = ux * Kwz;
    D[2][1][0] = uy * Kwx;
    D[0][1][2] = uy * Kwz;
    D[2][0][1] = uz * Kwx;
    D[0][2][1] = uz * Kwy;
    D[1][1][1] = ux * uy * uz;
    const float dx = D[2][0][0], dy = D[0][2][0], dz = D[0][0][2];
    D[2][2][0] = fmaf(Kwx, dy, fmaf(Kwy, dx, dx * dy));
    D[2][0][2] = fmaf(Kwx, dz, fmaf(Kwz, dx, dx * dz));
    D[0][2][2] = fmaf(Kwy, dz, fmaf(Kwz, dy, dy * dz));
    D[2][1][1] = -Kwx * uy * uz;
    D[1][2][1] = -ux * Kwy * uz;
    D[1][1][2] = -ux * uy * Kwz;
    D[1][2][2] = ux * Kwy * Kwz;
    D[2][1][2] = uy * Kwx * Kwz;
    D[2][2][1] = uz * Kwx * Kwy;
    D[2][2][2] = dx * Kwy * Kwz + dy * Kwx * Kwz + dz * Kwx * Kwy + dx * dy * Kwz +
                 dx * dz * Kwy + dy * dz * Kwx + dx * dy * dz;
    inverse27(D, ux, uy, uz, f);
}

}  // namespace lbm
