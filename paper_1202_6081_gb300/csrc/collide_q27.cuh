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
#include "vec2.cuh"

namespace lbm {

// slot (paper order) of the D3Q27 velocity with components (i-1, j-1, k-1)
__host__ __device__ constexpr int s27(int i, int j, int k) { return slot_of<27>(i - 1, j - 1, k - 1); }

// Relaxation rates as the collision consumes them: omega, -omega and
// 1 - omega per beta (0..3 unused), in the value type V (float, or f2 with
// both lanes equal).
template <typename V>
struct Rates27 {
    V w[27];
    V nw[27];
    V omw[27];
};

// 1-D shift of raw sums (m0, m1, m2) = (sum f, sum e f, sum e^2 f) of a line
// to central moments about u:  k1 = m1 - u m0,  k2 = m2 - 2 u m1 + u^2 m0.
// nu = -u.
template <typename V>
__device__ __forceinline__ void central_from_sums(V nu, V &m0, V &m1, V &m2) {
    const V k1 = vfma(nu, m0, m1);
    const V k2 = vfma(nu, m1 + k1, m2);
    m1 = k1;
    m2 = k2;
}

// raw sums of the line (a, b, c) = (f(-1), f(0), f(+1))
template <typename V>
__device__ __forceinline__ void sums(V a, V b, V c, V &s0, V &s1, V &s2) {
    const V ac = a + c;
    s0 = ac + b;
    s1 = c - a;
    s2 = ac;
}

// Inverse: central moments (k0, k1, k2) about u -> (f(-1), f(0), f(+1)).
template <typename V>
__device__ __forceinline__ void dist_from_central(V u, V k0, V k1, V k2, V &a, V &b, V &c) {
    const V half = splat<V>(0.5f);
    const V m1 = vfma(u, k0, k1);      // raw first moment
    const V m2 = vfma(u, k1 + m1, k2); // raw second moment
    b = k0 - m2;
    c = half * (m2 + m1);
    a = half * (m2 - m1);
}

// Relax the deviation central moments D[m][n][p] (= kappa - kappa^w,
// source included) in place.  drho = rho - 1.
//
// kEq: every rate from the trace on (omega_9 .. omega_26) is exactly 1 --
// the paper's tests and the benchmark relax all but the shear moments at 1.
// Then c~ = (1 - omega) c + omega c^at is c^at exactly (the FMA of a zero
// with c adds nothing, and a product with 1 is exact), so those moments are
// written from their attractors without reading c, and every operation of
// the forward sweeps that only fed a moment of order >= 3 (or the trace)
// becomes dead code for the compiler.  The same arithmetic as the general
// form; the results agree to rounding, not bit for bit, because the code
// generator fuses some packed multiply-add pairs differently in the two.
template <bool kEq, typename V>
__device__ __forceinline__ V relaxed(V omw, V c, V target) {
    if constexpr (kEq)
        return target;
    else
        return vfma(omw, c, target);
}

template <typename V, bool kEq = false>
__device__ __forceinline__ void relax27(V (&D)[3][3][3], V ux, V uy, V uz, V drho,
                                        const Rates27<V> &r) {
    const V third = splat<V>(1.0f / 3.0f), sixth = splat<V>(1.0f / 6.0f);
    const V half = splat<V>(0.5f), two = splat<V>(2.0f);
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V Kwx = third + ux2, Kwy = third + uy2, Kwz = third + uz2;

    // order 2, off-diagonal: attractor 0, kappa^w = u_i u_j
    D[1][1][0] = vfma(r.omw[4], D[1][1][0], r.nw[4] * (ux * uy));
    D[1][0][1] = vfma(r.omw[5], D[1][0][1], r.nw[5] * (ux * uz));
    D[0][1][1] = vfma(r.omw[6], D[0][1][1], r.nw[6] * (uy * uz));

    // order 2, diagonal: xx-yy -> 0, xx+yy-2zz -> 0, xx+yy+zz -> rho
    {
        const V xy = D[2][0][0] + D[0][2][0];
        V a = D[2][0][0] - D[0][2][0];
        V b = xy - two * D[0][0][2];
        V c = xy + D[0][0][2];
        const V uxy = ux2 + uy2;
        a = vfma(r.omw[7], a, r.nw[7] * (ux2 - uy2));
        b = vfma(r.omw[8], b, r.nw[8] * (uxy - two * uz2));
        c = kEq ? drho - (uxy + uz2) : vfma(r.omw[9], c, r.w[9] * (drho - (uxy + uz2)));
        const V c3 = c * third, b6 = b * sixth;
        const V cb = c3 + b6;
        D[2][0][0] = vfma(half, a, cb);
        D[0][2][0] = cb - half * a;
        D[0][0][2] = c3 - two * b6;
    }
    const V dxx = D[2][0][0], dyy = D[0][2][0], dzz = D[0][0][2];  // post-collision

    // order 3: attractors 0; kappa^w_xyy = -u_x Kw_y etc.
    {
        const V s = D[1][2][0] + D[1][0][2], t = D[1][2][0] - D[1][0][2];
        const V sn = kEq ? ux * (Kwy + Kwz) : vfma(r.omw[10], s, r.w[10] * (ux * (Kwy + Kwz)));
        const V tn = kEq ? ux * (Kwy - Kwz) : vfma(r.omw[13], t, r.w[13] * (ux * (Kwy - Kwz)));
        D[1][2][0] = half * (sn + tn);
        D[1][0][2] = half * (sn - tn);
    }
    {
        const V s = D[2][1][0] + D[0][1][2], t = D[2][1][0] - D[0][1][2];
        const V sn = kEq ? uy * (Kwx + Kwz) : vfma(r.omw[11], s, r.w[11] * (uy * (Kwx + Kwz)));
        const V tn = kEq ? uy * (Kwx - Kwz) : vfma(r.omw[14], t, r.w[14] * (uy * (Kwx - Kwz)));
        D[2][1][0] = half * (sn + tn);
        D[0][1][2] = half * (sn - tn);
    }
    {
        const V s = D[2][0][1] + D[0][2][1], t = D[2][0][1] - D[0][2][1];
        const V sn = kEq ? uz * (Kwx + Kwy) : vfma(r.omw[12], s, r.w[12] * (uz * (Kwx + Kwy)));
        const V tn = kEq ? uz * (Kwx - Kwy) : vfma(r.omw[15], t, r.w[15] * (uz * (Kwx - Kwy)));
        D[2][0][1] = half * (sn + tn);
        D[0][2][1] = half * (sn - tn);
    }
    D[1][1][1] = kEq ? ux * uy * uz : vfma(r.omw[16], D[1][1][1], r.w[16] * (ux * uy * uz));

    // order 4: xxyy, xxzz, yyzz -> products of the post-collision kappa~_ii
    {
        const V dA = vfma(Kwx, dyy, vfma(Kwy, dxx, dxx * dyy));  // kt_x kt_y - Kw_x Kw_y
        const V dB = vfma(Kwx, dzz, vfma(Kwz, dxx, dxx * dzz));
        const V dC = vfma(Kwy, dzz, vfma(Kwz, dyy, dyy * dzz));
        const V A = D[2][2][0], B = D[2][0][2], C = D[0][2][2];
        const V AB = A + B, dAB = dA + dB;
        const V p17 = kEq ? dAB + dC : vfma(r.omw[17], AB + C, r.w[17] * (dAB + dC));
        const V p18 = kEq ? dAB - two * dC : vfma(r.omw[18], AB - two * C, r.w[18] * (dAB - two * dC));
        const V p19 = kEq ? dA - dB : vfma(r.omw[19], A - B, r.w[19] * (dA - dB));
        const V ABn = third * (two * p17 + p18);
        D[0][2][2] = third * (p17 - p18);
        D[2][2][0] = half * (ABn + p19);
        D[2][0][2] = half * (ABn - p19);
    }
    // xxyz, xyyz, xyzz -> 0; kappa^w_xxyz = Kw_x u_y u_z etc.
    D[2][1][1] = relaxed<kEq>(r.omw[20], D[2][1][1], r.nw[20] * (Kwx * (uy * uz)));
    D[1][2][1] = relaxed<kEq>(r.omw[21], D[1][2][1], r.nw[21] * (Kwy * (ux * uz)));
    D[1][1][2] = relaxed<kEq>(r.omw[22], D[1][1][2], r.nw[22] * (Kwz * (ux * uy)));

    // order 5 -> 0; kappa^w_xyyzz = -u_x Kw_y Kw_z etc.
    D[1][2][2] = kEq ? ux * (Kwy * Kwz) : vfma(r.omw[23], D[1][2][2], r.w[23] * (ux * (Kwy * Kwz)));
    D[2][1][2] = kEq ? uy * (Kwx * Kwz) : vfma(r.omw[24], D[2][1][2], r.w[24] * (uy * (Kwx * Kwz)));
    D[2][2][1] = kEq ? uz * (Kwx * Kwy) : vfma(r.omw[25], D[2][2][1], r.w[25] * (uz * (Kwx * Kwy)));

    // order 6: xxyyzz -> kt_x kt_y kt_z;  kt_x kt_y kt_z - Kw_x Kw_y Kw_z
    {
        const V ktx = Kwx + dxx, kty = Kwy + dyy;
        // (Kwx + dxx)(Kwy + dyy)(Kwz + dzz) - Kwx Kwy Kwz
        //   = kt_x kt_y dzz + Kwz (kt_x dyy + Kwy dxx)
        const V dK = vfma(ktx * kty, dzz, Kwz * vfma(ktx, dyy, Kwy * dxx));
        D[2][2][2] = kEq ? dK : vfma(r.omw[26], D[2][2][2], r.w[26] * dK);
    }
}

// Forward transform of deviations f[slot] into central-moment space.
// Returns drho and u; D holds the central moments about u of the
// deviations, to which the caller adds the source.
template <typename V>
__device__ __forceinline__ void forward27(const V (&f)[27], V (&D)[3][3][3], V Fx, V Fy, V Fz,
                                          V &drho, V &ux, V &uy, V &uz) {
    // raw sums along x, then y, then z
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            sums(f[s27(0, j, k)], f[s27(1, j, k)], f[s27(2, j, k)], D[0][j][k], D[1][j][k],
                 D[2][j][k]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V s0, s1, s2;
            sums(D[m][0][k], D[m][1][k], D[m][2][k], s0, s1, s2);
            D[m][0][k] = s0;
            D[m][1][k] = s1;
            D[m][2][k] = s2;
        }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            V s0, s1, s2;
            sums(D[m][n][0], D[m][n][1], D[m][n][2], s0, s1, s2);
            D[m][n][0] = s0;
            D[m][n][1] = s1;
            D[m][n][2] = s2;
        }
    // D now holds raw moments of the deviations; the rest state has raw
    // moments (1, 0, 1/3, ...), so rho = 1 + drho and j = j_dev.
    const V half = splat<V>(0.5f);
    drho = D[0][0][0];
    const V inv_rho = vrcp(splat<V>(1.0f) + drho);
    ux = vfma(half, Fx, D[1][0][0]) * inv_rho;
    uy = vfma(half, Fy, D[0][1][0]) * inv_rho;
    uz = vfma(half, Fz, D[0][0][1]) * inv_rho;
    const V zero = splat<V>(0.0f);
    const V nux = zero - ux, nuy = zero - uy, nuz = zero - uz;
    // shift raw -> central about u, one axis at a time (the shifts commute)
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int p = 0; p < 3; ++p) central_from_sums(nux, D[0][n][p], D[1][n][p], D[2][n][p]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int p = 0; p < 3; ++p) central_from_sums(nuy, D[m][0][p], D[m][1][p], D[m][2][p]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) central_from_sums(nuz, D[m][n][0], D[m][n][1], D[m][n][2]);
}

// Inverse transform: deviation central moments about u -> deviations f[slot].
template <typename V>
__device__ __forceinline__ void inverse27(V (&D)[3][3][3], V ux, V uy, V uz, V (&f)[27]) {
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            V a, b, c;
            dist_from_central(uz, D[m][n][0], D[m][n][1], D[m][n][2], a, b, c);
            D[m][n][0] = a;
            D[m][n][1] = b;
            D[m][n][2] = c;
        }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V a, b, c;
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

// ---- lean variant for the two-cell kernels ------------------------------
//
// (1) The inverse sweeps leave out the factors 1/2 of dist_from_central: the
//     three inputs of every line share one power-of-two factor, so each
//     output f(i, j, k) comes out multiplied by G_i G_j G_k (G = 2, 1, 2 for
//     e = -1, 0, +1), exactly, and the kernel folds 1 / (G_i G_j G_k) into
//     the one multiplication it applies at the store anyway (FP32: exact
//     powers of two, so the stored values are bit-identical).
// (2) For storage of s = (f - w) / w the forward sweeps fold the weights in:
//     w = W_i W_j W_k / 216 with W = (1, 4, 1), so a + 4 b + c along each
//     axis gives 216 times the moments of the deviations with no per-value
//     multiplication.  The relaxation is linear in the pre-collision moments
//     (c~ = (1 - omega) c + omega c^eq), so dividing 1 - omega by 216 on the
//     host (packed_rates) relaxes the scaled moments correctly; only the
//     invariant moments (orders 0 and 1) are scaled back explicitly.

// G_i G_j G_k of slot q
__host__ __device__ constexpr int g27(int q) {
    return (q27_e(q, 0) ? 2 : 1) * (q27_e(q, 1) ? 2 : 1) * (q27_e(q, 2) ? 2 : 1);
}

template <typename V>
__device__ __forceinline__ void dist_from_central_g(V u, V k0, V k1, V k2, V &a, V &b, V &c) {
    const V m1 = vfma(u, k0, k1);
    const V m2 = vfma(u, k1 + m1, k2);
    b = k0 - m2;
    c = m2 + m1;
    a = m2 - m1;
}

template <typename V>
__device__ __forceinline__ void inverse27_g(V (&D)[3][3][3], V ux, V uy, V uz, V (&f)[27]) {
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            V a, b, c;
            dist_from_central_g(uz, D[m][n][0], D[m][n][1], D[m][n][2], a, b, c);
            D[m][n][0] = a;
            D[m][n][1] = b;
            D[m][n][2] = c;
        }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V a, b, c;
            dist_from_central_g(uy, D[m][0][k], D[m][1][k], D[m][2][k], a, b, c);
            D[m][0][k] = a;
            D[m][1][k] = b;
            D[m][2][k] = c;
        }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dist_from_central_g(ux, D[0][j][k], D[1][j][k], D[2][j][k], f[s27(0, j, k)],
                                f[s27(1, j, k)], f[s27(2, j, k)]);
}

// weighted raw sums of the line (a, b, c) = (s(-1), s(0), s(+1)), weights (1, 4, 1)
template <typename V>
__device__ __forceinline__ void sums_w(V a, V b, V c, V &s0, V &s1, V &s2) {
    const V ac = a + c;
    s0 = vfma(splat<V>(4.0f), b, ac);
    s1 = c - a;
    s2 = ac;
}

// Forward transform of weight-scaled values s (f - w = w s): D = 216 x the
// central moments of the deviations for orders >= 2, the true ones for
// orders 0 and 1; drho and u as in forward27.
template <typename V>
__device__ __forceinline__ void forward27_w(const V (&s)[27], V (&D)[3][3][3], V Fx, V Fy, V Fz,
                                            V &drho, V &ux, V &uy, V &uz) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            sums_w(s[s27(0, j, k)], s[s27(1, j, k)], s[s27(2, j, k)], D[0][j][k], D[1][j][k],
                   D[2][j][k]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V s0, s1, s2;
            sums_w(D[m][0][k], D[m][1][k], D[m][2][k], s0, s1, s2);
            D[m][0][k] = s0;
            D[m][1][k] = s1;
            D[m][2][k] = s2;
        }
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            V s0, s1, s2;
            sums_w(D[m][n][0], D[m][n][1], D[m][n][2], s0, s1, s2);
            D[m][n][0] = s0;
            D[m][n][1] = s1;
            D[m][n][2] = s2;
        }
    const V half = splat<V>(0.5f), inv216 = splat<V>(1.0f / 216.0f);
    drho = D[0][0][0] * inv216;
    const V inv_rho = vrcp(splat<V>(1.0f) + drho);
    ux = vfma(D[1][0][0], inv216, half * Fx) * inv_rho;
    uy = vfma(D[0][1][0], inv216, half * Fy) * inv_rho;
    uz = vfma(D[0][0][1], inv216, half * Fz) * inv_rho;
    const V zero = splat<V>(0.0f);
    const V nux = zero - ux, nuy = zero - uy, nuz = zero - uz;
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
        for (int p = 0; p < 3; ++p) central_from_sums(nux, D[0][n][p], D[1][n][p], D[2][n][p]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int p = 0; p < 3; ++p) central_from_sums(nuy, D[m][0][p], D[m][1][p], D[m][2][p]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n) central_from_sums(nuz, D[m][n][0], D[m][n][1], D[m][n][2]);
    // the collision invariants are not relaxed: back to true scale
    D[0][0][0] = drho;
    D[1][0][0] = D[1][0][0] * inv216;
    D[0][1][0] = D[0][1][0] * inv216;
    D[0][0][1] = D[0][0][1] * inv216;
}

// The collision of collide27 with outputs G_i G_j G_k f~ (see (1) above);
// kWeighted: inputs are weight-scaled values s and r.omw holds
// (1 - omega) / 216 (see (2) above).
// u_out: the velocity (with the F/2 shift) of Eq. velocitycalculation.
template <typename V, bool kWeighted, bool kEq = false>
__device__ __forceinline__ void collide27_g(V (&f)[27], V Fx, V Fy, V Fz, const Rates27<V> &r,
                                            V &ux, V &uy, V &uz) {
    V D[3][3][3];
    V drho;
    if constexpr (kWeighted)
        forward27_w(f, D, Fx, Fy, Fz, drho, ux, uy, uz);
    else
        forward27(f, D, Fx, Fy, Fz, drho, ux, uy, uz);
    D[1][0][0] = D[1][0][0] + Fx;
    D[0][1][0] = D[0][1][0] + Fy;
    D[0][0][1] = D[0][0][1] + Fz;
    relax27<V, kEq>(D, ux, uy, uz, drho, r);
    inverse27_g(D, ux, uy, uz, f);
}
template <typename V, bool kWeighted, bool kEq = false>
__device__ __forceinline__ void collide27_g(V (&f)[27], V Fx, V Fy, V Fz, const Rates27<V> &r) {
    V ux, uy, uz;
    collide27_g<V, kWeighted, kEq>(f, Fx, Fy, Fz, r, ux, uy, uz);
}

// One cell (or a pair of cells, V = f2): pre-collision deviations in,
// post-collision deviations out (both f - w, slot order).
template <typename V>
__device__ __forceinline__ void collide27(V (&f)[27], V Fx, V Fy, V Fz, const Rates27<V> &r,
                                          V &ux, V &uy, V &uz) {
    V D[3][3][3];
    V drho;
    forward27(f, D, Fx, Fy, Fz, drho, ux, uy, uz);
    // The sweeps produced the central moments of the deviations; those of
    // the rest state are handled in closed form inside relax27, so D is
    // d = kappa - kappa^w.  Add the source's central moments: F at first
    // order, zero elsewhere (Eq. discretecentralsources).
    D[1][0][0] = D[1][0][0] + Fx;
    D[0][1][0] = D[0][1][0] + Fy;
    D[0][0][1] = D[0][0][1] + Fz;
    relax27(D, ux, uy, uz, drho, r);
    inverse27(D, ux, uy, uz, f);
}
template <typename V>
__device__ __forceinline__ void collide27(V (&f)[27], V Fx, V Fy, V Fz, const Rates27<V> &r) {
    V ux, uy, uz;
    collide27<V>(f, Fx, Fy, Fz, r, ux, uy, uz);
}

// The change the collision makes, d = f~ - f (source included), for the
// incremental update f~ = f + d: the inverse transform is linear in the
// moments for a given u, and maps the pre-collision moments back to f, so
// d = Inv(D~ - D) with D the pre-collision moments (before the source).
__device__ __forceinline__ void collide27_delta(const float (&f)[27], float Fx, float Fy, float Fz,
                                                const Rates27<float> &r, float (&d)[27]) {
    float D[3][3][3], D0[3][3][3];
    float drho, ux, uy, uz;
    forward27(f, D, Fx, Fy, Fz, drho, ux, uy, uz);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int p = 0; p < 3; ++p) D0[m][n][p] = D[m][n][p];
    D[1][0][0] = D[1][0][0] + Fx;
    D[0][1][0] = D[0][1][0] + Fy;
    D[0][0][1] = D[0][0][1] + Fz;
    relax27(D, ux, uy, uz, drho, r);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
#pragma unroll
            for (int p = 0; p < 3; ++p) D[m][n][p] = D[m][n][p] - D0[m][n][p];
    inverse27(D, ux, uy, uz, d);
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
    inverse27<float>(D, ux, uy, uz, f);
}

}  // namespace lbm
