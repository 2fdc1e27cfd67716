// D3Q15 central-moment collision with forcing, in registers, on deviations.
//
// D3Q15 has no tensor-product structure, so the collision follows the
// cascade of App. G directly: raw moments of the pre-collision state, raw
// source moments (App. C), the kernels g_4..g_14 in order (each relaxing one
// central moment -- xy, xz, yz, xx-yy, xx+yy-2zz, xx+yy+zz, xyy, xxy, xxz,
// xyz, xxyy -- toward its attractor, with the lower kernels feeding the
// higher ones), then f~ = f + K.g + S with K the D3Q15 basis and
// S = K D^-1 m^s the source of App. G.
//
// GB300 form: templated on the value type (float, or f2 = two neighbouring
// cells in packed f32x2 arithmetic), and both directions between the
// populations and the moments go by sign patterns instead of 15 x 15 and
// 15 x 11 products: on the 8 corners (sx, sy, sz) every basis vector and
// every raw moment the cascade needs is one of 1, sx, sy, sz, sx sy, sx sz,
// sy sz, sx sy sz times a constant, so the moment sums and the 8 corner
// increments are three-level butterflies; each axis pair (+-x etc.) enters
// as a sum and a difference (even and odd parts).
//
// Precision: the state is carried as deviations from the weights
// (2/9, 1/9, 1/72).  The weights' raw moments are 1 (mass), 1/3 (xx, yy, zz)
// and 1/9 (xxyy), zero otherwise; wherever such a constant meets its
// attractor (rho, kappa~_xx kappa~_yy) the pair is cancelled analytically.
#pragma once

#include "lattice.cuh"
#include "vec2.cuh"

namespace lbm {

// D3Q15 basis vector K_beta evaluated at velocity slot a (App. G).
__host__ __device__ constexpr int k15(int b, int a) {
    const int x = q15_e(a, 0), y = q15_e(a, 1), z = q15_e(a, 2);
    const int n = x * x + y * y + z * z;
    switch (b) {
        case 0: return 1;
        case 1: return x;
        case 2: return y;
        case 3: return z;
        case 4: return x * y;
        case 5: return x * z;
        case 6: return y * z;
        case 7: return x * x - y * y;
        case 8: return x * x + y * y - 2 * z * z;
        case 9: return n - 2;
        case 10: return (5 * n - 13) * x;
        case 11: return (5 * n - 13) * y;
        case 12: return (5 * n - 13) * z;
        case 13: return x * y * z;
        default: return 30 * (x * x * y * y + x * x * z * z + y * y * z * z) - 40 * n + 32;
    }
}

// App. G prefactors 1/k_beta of the kernels g_4..g_14 (omega_beta / k_beta).
__host__ __device__ constexpr float k15_inv(int b) {
    return b <= 6 ? 0.125f
         : b == 7 ? 0.25f
         : b == 8 ? 1.0f / 12.0f
         : b == 9 ? 1.0f / 18.0f
         : b <= 12 ? 0.0625f
         : b == 13 ? 0.125f
                   : 0.0625f;
}

// omega_beta / k_beta per beta, in the value type V.
template <typename V>
struct Rates15 {
    V w[15];
};

// Projections m^s_beta = <K_beta|S> of the source (App. G), beta = 0..14.
template <typename V>
__device__ __forceinline__ void source_projections15(V Fx, V Fy, V Fz, V ux, V uy, V uz,
                                                     V (&m)[15]) {
    const V two = splat<V>(2.0f), three = splat<V>(3.0f), five = splat<V>(5.0f);
    const V m4 = splat<V>(-4.0f), m13 = splat<V>(-13.0f);
    m[0] = splat<V>(0.0f);
    m[1] = Fx;
    m[2] = Fy;
    m[3] = Fz;
    m[4] = vfma(Fx, uy, Fy * ux);
    m[5] = vfma(Fx, uz, Fz * ux);
    m[6] = vfma(Fy, uz, Fz * uy);
    const V fux = Fx * ux, fuy = Fy * uy, fuz = Fz * uz;
    m[7] = two * (fux - fuy);
    m[8] = two * ((fux + fuy) - two * fuz);
    m[9] = two * (fux + fuy + fuz);
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    m[10] = vfma(five, vfma(Fx, vfma(three, ux2, uy2 + uz2), two * ux * (fuy + fuz)), m13 * Fx);
    m[11] = vfma(five, vfma(Fy, vfma(three, uy2, ux2 + uz2), two * uy * (fux + fuz)), m13 * Fy);
    m[12] = vfma(five, vfma(Fz, vfma(three, uz2, ux2 + uy2), two * uz * (fux + fuy)), m13 * Fz);
    m[13] = vfma(Fx, uy * uz, vfma(Fy, ux * uz, Fz * (ux * uy)));
    m[14] = splat<V>(20.0f) * vfma(fux, vfma(three, uy2 + uz2, m4),
                                   vfma(fuy, vfma(three, ux2 + uz2, m4),
                                        fuz * vfma(three, ux2 + uy2, m4)));
}

// The 8 sign-pattern sums over the corners (sx, sy, sz) of v: sum of v,
// of sx v, sy v, sz v, sx sy v, sx sz v, sy sz v and sx sy sz v, as a
// three-level butterfly (24 additions instead of 8 per pattern); and the
// axis pairs as sums a_i = v(+e_i) + v(-e_i) and differences d_i.
template <typename V>
__device__ __forceinline__ void corner_axis_sums15(const V (&v)[15], V &C, V &Cx, V &Cy, V &Cz,
                                                   V &Cxy, V &Cxz, V &Cyz, V &Cxyz, V &ax, V &ay,
                                                   V &az, V &dx, V &dy, V &dz) {
    // level 1 over sz: S/D[i][j] at sx = i ? -1 : +1, sy = j ? -1 : +1
    V S[2][2], D[2][2];
    static_for<4>([&](auto ij) {
        constexpr int i = decltype(ij)::value >> 1, j = decltype(ij)::value & 1;
        constexpr int sx = i ? -1 : 1, sy = j ? -1 : 1;
        const V up = v[slot_of<15>(sx, sy, 1)], dn = v[slot_of<15>(sx, sy, -1)];
        S[i][j] = up + dn;
        D[i][j] = up - dn;
    });
    // level 2 over sy: patterns 1, sy, sz, sy sz at sx = +1 (index 0) and -1
    V c1[2], cy[2], cz[2], cyz[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        c1[i] = S[i][0] + S[i][1];
        cy[i] = S[i][0] - S[i][1];
        cz[i] = D[i][0] + D[i][1];
        cyz[i] = D[i][0] - D[i][1];
    }
    // level 3 over sx
    C = c1[0] + c1[1];
    Cx = c1[0] - c1[1];
    Cy = cy[0] + cy[1];
    Cxy = cy[0] - cy[1];
    Cz = cz[0] + cz[1];
    Cxz = cz[0] - cz[1];
    Cyz = cyz[0] + cyz[1];
    Cxyz = cyz[0] - cyz[1];
    constexpr int px = slot_of<15>(1, 0, 0), mx = slot_of<15>(-1, 0, 0);
    constexpr int py = slot_of<15>(0, 1, 0), my = slot_of<15>(0, -1, 0);
    constexpr int pz = slot_of<15>(0, 0, 1), mz = slot_of<15>(0, 0, -1);
    ax = v[px] + v[mx];
    ay = v[py] + v[my];
    az = v[pz] + v[mz];
    dx = v[px] - v[mx];
    dy = v[py] - v[my];
    dz = v[pz] - v[mz];
}

// Signed sums of the deviations over the index sets of App. G (the raw
// moments the cascade needs).  D3Q15 has no xy, xz or yz edges, so every
// mixed moment lives on the corners alone and is one sign pattern there.
template <typename V>
__device__ __forceinline__ void sums15(const V (&f)[15], V &drho, V &jx, V &jy, V &jz, V &kxy,
                                       V &kxz, V &kyz, V &kxx, V &kyy, V &kzz, V &kxyy, V &kxxy,
                                       V &kxxz, V &kxyz, V &kxxyy) {
    V C, ax, ay, az, dx, dy, dz;
    corner_axis_sums15(f, C, kxyy, kxxy, kxxz, kxy, kxz, kyz, kxyz, ax, ay, az, dx, dy, dz);
    kxxyy = C;
    jx = dx + kxyy;
    jy = dy + kxxy;
    jz = dz + kxxz;
    kxx = ax + C;
    kyy = ay + C;
    kzz = az + C;
    drho = ((f[0] + C) + ax) + (ay + az);
}

// The cascade on deviation raw moments; returns u and g[4..14].  The rates
// carry the App. G prefactors: r.w[beta] = omega_beta / k_beta.
template <typename V>
__device__ __forceinline__ void kernels15(const V (&f)[15], V Fx, V Fy, V Fz, const Rates15<V> &r,
                                          V &ux, V &uy, V &uz, V (&g)[15]) {
    const V zero = splat<V>(0.0f);
    V drho, jx, jy, jz, kxy, kxz, kyz, kxx, kyy, kzz, kxyy, kxxy, kxxz, kxyz, kxxyy;
    sums15(f, drho, jx, jy, jz, kxy, kxz, kyz, kxx, kyy, kzz, kxyy, kxxy, kxxz, kxyz, kxxyy);
    const V one = splat<V>(1.0f), half = splat<V>(0.5f), two = splat<V>(2.0f);
    const V three = splat<V>(3.0f), eighth = splat<V>(0.125f);
    const V rho = one + drho;
    const V inv_rho = vrcp(rho);
    ux = vfma(half, Fx, jx) * inv_rho;
    uy = vfma(half, Fy, jy) * inv_rho;
    uz = vfma(half, Fz, jz) * inv_rho;
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;
    // raw source moments (App. C); eta' = kappa' + sigma' as deviations
    const V sx = Fx, sy = Fy, sz = Fz;
    const V fux = Fx * ux, fuy = Fy * uy, fuz = Fz * uz;
    const V exy = kxy + vfma(Fx, uy, Fy * ux);
    const V exz = kxz + vfma(Fx, uz, Fz * ux);
    const V eyz = kyz + vfma(Fy, uz, Fz * uy);
    const V exx = vfma(two, fux, kxx);
    const V eyy = vfma(two, fuy, kyy);
    const V ezz = vfma(two, fuz, kzz);
    const V exyy = kxyy + vfma(Fx, uy2, two * fuy * ux);
    const V exxy = kxxy + vfma(Fy, ux2, two * fux * uy);
    const V exxz = kxxz + vfma(Fz, ux2, two * fux * uz);
    const V exyz = kxyz + vfma(Fx, uyz, vfma(Fy, uxz, Fz * uxy));
    const V exxyy = kxxyy + two * vfma(fux, uy2, fuy * ux2);
    const V third = splat<V>(1.0f / 3.0f);
    const V Exx = third + exx, Eyy = third + eyy;  // full eta'_xx, eta'_yy

    const V s_u = vfma(sx, ux, vfma(sy, uy, sz * uz));
#pragma unroll
    for (int b = 0; b < 4; ++b) g[b] = zero;
    g[4] = r.w[4] * (vfma(rho, uxy, half * vfma(sx, uy, sy * ux)) - exy);
    g[5] = r.w[5] * (vfma(rho, uxz, half * vfma(sx, uz, sz * ux)) - exz);
    g[6] = r.w[6] * (vfma(rho, uyz, half * vfma(sy, uz, sz * uy)) - eyz);
    g[7] = r.w[7] * (vfma(rho, ux2 - uy2, fux - fuy) - (exx - eyy));
    g[8] = r.w[8] * (vfma(rho, (ux2 + uy2) - two * uz2, (fux + fuy) - two * fuz) -
                     ((exx + eyy) - two * ezz));
    // -(eta'_xx + eta'_yy + eta'_zz) + rho = -(deviation sum) - 1 + rho
    g[9] = r.w[9] * (vfma(rho, ux2 + uy2 + uz2, s_u + drho) - (exx + eyy + ezz));
    g[10] = vfma(r.w[10],
                 vfma(two * uy, exy, ux * Eyy) -
                     vfma(two * rho * ux, uy2, vfma(half * sx, uy2, sy * uy * ux)) - exyy,
                 vfma(uy, g[4], eighth * ux * vfma(three, g[9], g[8] - g[7])));
    g[11] = vfma(r.w[11],
                 vfma(two * ux, exy, uy * Exx) -
                     vfma(two * rho * ux2, uy, vfma(half * sy, ux2, sx * uxy)) - exxy,
                 vfma(ux, g[4], eighth * uy * vfma(three, g[9], g[8] + g[7])));
    g[12] = vfma(r.w[12],
                 vfma(two * ux, exz, uz * Exx) -
                     vfma(two * rho * ux2, uz, vfma(half * sz, ux2, sx * uxz)) - exxz,
                 vfma(ux, g[5], eighth * uz * vfma(three, g[9], g[8] + g[7])));
    g[13] = vfma(r.w[13],
                 vfma(ux, eyz, vfma(uy, exz, uz * exy)) -
                     vfma(two * rho, ux * uyz, half * vfma(sx, uyz, vfma(sy, uxz, sz * uxy))) -
                     exyz,
                 vfma(uz, g[4], vfma(uy, g[5], ux * g[6])));
    // post-collision kappa~_xx, kappa~_yy as deviations from 1/3
    const V six = splat<V>(6.0f);
    const V dkx = vfma(six, g[9], exx + two * (g[7] + g[8])) - vfma(rho, ux2, fux);
    const V dky = vfma(six, g[9], eyy + two * (g[8] - g[7])) - vfma(rho, uy2, fuy);
    // -eta'_xxyy + kappa~_xx kappa~_yy = -dev_xxyy + (dkx + dky)/3 + dkx dky
    const V br14 = vfma(two * ux, exyy, two * uy * exxy) - vfma(ux2, Eyy, uy2 * Exx) -
                   splat<V>(4.0f) * uxy * exy + vfma(dkx + dky, third, dkx * dky) +
                   vfma(three * rho, ux2 * uy2, vfma(sx, ux * uy2, sy * uy * ux2)) - exxyy;
    g[14] = vfma(r.w[14], br14,
                 vfma(splat<V>(-2.0f) * uxy, g[4],
                      vfma(eighth * (ux2 - uy2), g[7],
                           vfma(splat<V>(-0.125f) * (ux2 + uy2), g[8],
                                vfma(vfma(splat<V>(-0.375f), ux2 + uy2, splat<V>(-0.5f)), g[9],
                                     two * vfma(ux, g[10], uy * g[11]))))));
}

// kernels15 with F = 0 written out (no force anywhere, the source term
// vanishes): the same cascade with every force product dropped, about 60
// fewer operations per cell; the sums are shared with kernels15.
template <typename V>
__device__ __forceinline__ void kernels15_unforced(const V (&f)[15], const Rates15<V> &r, V &ux,
                                                   V &uy, V &uz, V (&g)[15]) {
    const V zero = splat<V>(0.0f);
    V drho, jx, jy, jz, kxy, kxz, kyz, kxx, kyy, kzz, kxyy, kxxy, kxxz, kxyz, kxxyy;
    sums15(f, drho, jx, jy, jz, kxy, kxz, kyz, kxx, kyy, kzz, kxyy, kxxy, kxxz, kxyz, kxxyy);
    const V one = splat<V>(1.0f), two = splat<V>(2.0f);
    const V three = splat<V>(3.0f), eighth = splat<V>(0.125f), third = splat<V>(1.0f / 3.0f);
    const V rho = one + drho;
    const V inv_rho = vrcp(rho);
    ux = jx * inv_rho;
    uy = jy * inv_rho;
    uz = jz * inv_rho;
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;
    const V Exx = third + kxx, Eyy = third + kyy;
#pragma unroll
    for (int b = 0; b < 4; ++b) g[b] = zero;
    g[4] = r.w[4] * (rho * uxy - kxy);
    g[5] = r.w[5] * (rho * uxz - kxz);
    g[6] = r.w[6] * (rho * uyz - kyz);
    g[7] = r.w[7] * vfma(rho, ux2 - uy2, kyy - kxx);
    g[8] = r.w[8] * vfma(rho, (ux2 + uy2) - two * uz2, two * kzz - (kxx + kyy));
    g[9] = r.w[9] * (vfma(rho, ux2 + uy2 + uz2, drho) - (kxx + kyy + kzz));
    const V rho2 = two * rho;
    g[10] = vfma(r.w[10], vfma(two * uy, kxy, ux * Eyy) - (rho2 * ux) * uy2 - kxyy,
                 vfma(uy, g[4], eighth * ux * vfma(three, g[9], g[8] - g[7])));
    g[11] = vfma(r.w[11], vfma(two * ux, kxy, uy * Exx) - (rho2 * ux2) * uy - kxxy,
                 vfma(ux, g[4], eighth * uy * vfma(three, g[9], g[8] + g[7])));
    g[12] = vfma(r.w[12], vfma(two * ux, kxz, uz * Exx) - (rho2 * ux2) * uz - kxxz,
                 vfma(ux, g[5], eighth * uz * vfma(three, g[9], g[8] + g[7])));
    g[13] = vfma(r.w[13], vfma(ux, kyz, vfma(uy, kxz, uz * kxy)) - rho2 * (ux * uyz) - kxyz,
                 vfma(uz, g[4], vfma(uy, g[5], ux * g[6])));
    const V six = splat<V>(6.0f);
    const V dkx = vfma(six, g[9], kxx + two * (g[7] + g[8])) - rho * ux2;
    const V dky = vfma(six, g[9], kyy + two * (g[8] - g[7])) - rho * uy2;
    const V br14 = vfma(two * ux, kxyy, two * uy * kxxy) - vfma(ux2, Eyy, uy2 * Exx) -
                   splat<V>(4.0f) * uxy * kxy + vfma(dkx + dky, third, dkx * dky) +
                   (three * rho) * (ux2 * uy2) - kxxyy;
    g[14] = vfma(r.w[14], br14,
                 vfma(splat<V>(-2.0f) * uxy, g[4],
                      vfma(eighth * (ux2 - uy2), g[7],
                           vfma(splat<V>(-0.125f) * (ux2 + uy2), g[8],
                                vfma(vfma(splat<V>(-0.375f), ux2 + uy2, splat<V>(-0.5f)), g[9],
                                     two * vfma(ux, g[10], uy * g[11]))))));
}

// Add K.g (and with kSource the source S of App. G, from its projections m)
// to the deviations f, by sign patterns (see the file comment).
template <typename V, bool kSource>
__device__ __forceinline__ void update15(V (&f)[15], const V (&g)[15], const V (&m)[15]) {
    const V two = splat<V>(2.0f), eight = splat<V>(8.0f), m8 = splat<V>(-8.0f);
    // rest: K.g = -2 g9 + 32 g14;  S = (3 m0 - 5 m9 + m14) / 45
    V rest = vfma(splat<V>(32.0f), g[14], splat<V>(-2.0f) * g[9]);
    // axis pairs: even part E, odd part O
    const V g914 = vfma(eight, g[14], g[9]);
    V Ex = (g[7] + g[8]) - g914;
    V Ey = (g[8] - g[7]) - g914;
    V Ez = splat<V>(-2.0f) * g[8] - g914;
    V Ox = m8 * g[10], Oy = m8 * g[11], Oz = m8 * g[12];
    // corners: c0 + sx cx + sy cy + sz cz + sx sy cxy + sx sz cxz + sy sz cyz
    //          + sx sy sz cxyz
    V c0 = vfma(two, g[14], g[9]);
    V cx = two * g[10], cy = two * g[11], cz = two * g[12];
    V cxy = g[4], cxz = g[5], cyz = g[6], cxyz = g[13];
    if constexpr (kSource) {
        const V i180 = splat<V>(1.0f / 180.0f), i720 = splat<V>(1.0f / 720.0f);
        rest = vfma(splat<V>(1.0f / 45.0f), vfma(splat<V>(-5.0f), m[9], m[14]), rest);
        const V ev = vfma(splat<V>(10.0f), m[9], m[14]);
        Ex = vfma(i180, vfma(splat<V>(45.0f), m[7], splat<V>(15.0f) * m[8]) - ev, Ex);
        Ey = vfma(i180, vfma(splat<V>(-45.0f), m[7], splat<V>(15.0f) * m[8]) - ev, Ey);
        Ez = vfma(i180, splat<V>(-30.0f) * m[8] - ev, Ez);
        Ox = vfma(i180, vfma(splat<V>(18.0f), m[1], splat<V>(-9.0f) * m[10]), Ox);
        Oy = vfma(i180, vfma(splat<V>(18.0f), m[2], splat<V>(-9.0f) * m[11]), Oy);
        Oz = vfma(i180, vfma(splat<V>(18.0f), m[3], splat<V>(-9.0f) * m[12]), Oz);
        c0 = vfma(i720, vfma(splat<V>(40.0f), m[9], m[14]), c0);
        cx = vfma(i720, vfma(splat<V>(72.0f), m[1], splat<V>(9.0f) * m[10]), cx);
        cy = vfma(i720, vfma(splat<V>(72.0f), m[2], splat<V>(9.0f) * m[11]), cy);
        cz = vfma(i720, vfma(splat<V>(72.0f), m[3], splat<V>(9.0f) * m[12]), cz);
        const V eighth = splat<V>(0.125f);
        cxy = vfma(eighth, m[4], cxy);
        cxz = vfma(eighth, m[5], cxz);
        cyz = vfma(eighth, m[6], cyz);
        cxyz = vfma(eighth, m[13], cxyz);
    }
    f[0] = f[0] + rest;
    f[1] = f[1] + (Ex + Ox);  // (+1, 0, 0)
    f[2] = f[2] + (Ex - Ox);  // (-1, 0, 0)
    f[3] = f[3] + (Ey + Oy);
    f[4] = f[4] + (Ey - Oy);
    f[5] = f[5] + (Ez + Oz);
    f[6] = f[6] + (Ez - Oz);
    // butterflies over sz, then sy, then sx (index 0: sz = +1, 1: sz = -1)
    V A[2], Bx[2], By[2], Bxy[2];
    A[0] = c0 + cz;
    A[1] = c0 - cz;
    Bx[0] = cx + cxz;
    Bx[1] = cx - cxz;
    By[0] = cy + cyz;
    By[1] = cy - cyz;
    Bxy[0] = cxy + cxyz;
    Bxy[1] = cxy - cxyz;
    static_for<8>([&](auto ic) {
        constexpr int a = 7 + decltype(ic)::value;
        constexpr int x = q15_e(a, 0), y = q15_e(a, 1), z = q15_e(a, 2);
        constexpr int k = z > 0 ? 0 : 1;
        const V P = y > 0 ? A[k] + By[k] : A[k] - By[k];
        const V R = y > 0 ? Bx[k] + Bxy[k] : Bx[k] - Bxy[k];
        f[a] = f[a] + (x > 0 ? P + R : P - R);
    });
}

// One cell (or a pair, V = f2): deviations in, post-collision deviations
// out.  with_source = false (no force anywhere) takes the force-free cascade
// and skips S.
// u_out: the velocity (with the F/2 shift).
template <typename V>
__device__ __forceinline__ void collide15(V (&f)[15], V Fx, V Fy, V Fz, const Rates15<V> &r,
                                          bool with_source, V &ux, V &uy, V &uz) {
    V g[15];
    V m[15];
    if (with_source) {
        kernels15(f, Fx, Fy, Fz, r, ux, uy, uz, g);
        source_projections15(Fx, Fy, Fz, ux, uy, uz, m);
        update15<V, true>(f, g, m);
    } else {
        kernels15_unforced(f, r, ux, uy, uz, g);
        update15<V, false>(f, g, m);
    }
}
template <typename V>
__device__ __forceinline__ void collide15(V (&f)[15], V Fx, V Fy, V Fz, const Rates15<V> &r,
                                          bool with_source) {
    V ux, uy, uz;
    collide15<V>(f, Fx, Fy, Fz, r, with_source, ux, uy, uz);
}

// The change the collision makes, d = K.g + S (Eq. cascadedcollision1), for
// the incremental update f~ = f + d: the update applied to zeros.
__device__ __forceinline__ void collide15_delta(const float (&f)[15], float Fx, float Fy,
                                                float Fz, const Rates15<float> &r, bool with_source,
                                                float (&d)[15]) {
    float g[15], m[15], ux, uy, uz;
#pragma unroll
    for (int a = 0; a < 15; ++a) d[a] = 0.0f;
    if (with_source) {
        kernels15(f, Fx, Fy, Fz, r, ux, uy, uz, g);
        source_projections15(Fx, Fy, Fz, ux, uy, uz, m);
        update15<float, true>(d, g, m);
    } else {
        kernels15_unforced(f, r, ux, uy, uz, g);
        update15<float, false>(d, g, m);
    }
}

// Deviations of f = f^at(rho, u) - S/2: one collision with every omega = 1
// and no force, from a state of the right mass and momentum
// (w (rho + 3 rho u.e)), then minus half the source at (F, u).
__device__ __forceinline__ void equilibrium15(float drho, float ux, float uy, float uz, float Fx,
                                              float Fy, float Fz, float (&f)[15]) {
    const float rho = 1.0f + drho;
    static_for<15>([&](auto ia) {
        constexpr int a = decltype(ia)::value;
        constexpr int cx = q15_e(a, 0), cy = q15_e(a, 1), cz = q15_e(a, 2);
        const float eu = cx * ux + cy * uy + cz * uz;
        f[a] = float(weight<15>(a)) * (drho + 3.0f * rho * eu);
    });
    Rates15<float> ones;
#pragma unroll
    for (int b = 0; b < 15; ++b) ones.w[b] = k15_inv(b);
    float g[15], ux0, uy0, uz0, m[15];
    kernels15<float>(f, 0.0f, 0.0f, 0.0f, ones, ux0, uy0, uz0, g);
    update15<float, false>(f, g, m);
    // minus half the source at (F, u): the update with g = 0 adds S alone
    float S[15], zg[15];
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        S[a] = 0.0f;
        zg[a] = 0.0f;
    }
    source_projections15<float>(Fx, Fy, Fz, ux, uy, uz, m);
    update15<float, true>(S, zg, m);
#pragma unroll
    for (int a = 0; a < 15; ++a) f[a] = f[a] - 0.5f * S[a];
}

}  // namespace lbm
