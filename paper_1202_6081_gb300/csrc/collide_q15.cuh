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
// Precision: the state is carried as deviations from the weights
// (2/9, 1/9, 1/72).  The weights' raw moments are 1 (mass), 1/3 (xx, yy, zz)
// and 1/9 (xxyy), zero otherwise; wherever such a constant meets its
// attractor (rho, kappa~_xx kappa~_yy) the pair is cancelled analytically.
#pragma once

#include "lattice.cuh"

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

// <K_beta|K_beta> on D3Q15
__host__ __device__ constexpr int d15(int b) {
    int s = 0;
    for (int a = 0; a < 15; ++a) s += k15(b, a) * k15(b, a);
    return s;
}

struct RelaxRates15 {
    float w[15];
};

// Source S_alpha = sum_beta K_beta(e_alpha) m^s_beta / D_beta with the
// projections m^s_beta of App. G.
__device__ __forceinline__ void source15(float Fx, float Fy, float Fz, float ux, float uy,
                                         float uz, float (&S)[15]) {
    float m[15];
    m[0] = 0.0f;
    m[1] = Fx;
    m[2] = Fy;
    m[3] = Fz;
    m[4] = Fx * uy + Fy * ux;
    m[5] = Fx * uz + Fz * ux;
    m[6] = Fy * uz + Fz * uy;
    const float fux = Fx * ux, fuy = Fy * uy, fuz = Fz * uz;
    m[7] = 2.0f * (fux - fuy);
    m[8] = 2.0f * (fux + fuy - 2.0f * fuz);
    m[9] = 2.0f * (fux + fuy + fuz);
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    m[10] = 5.0f * (Fx * (3.0f * ux2 + uy2 + uz2) + 2.0f * ux * (fuy + fuz)) - 13.0f * Fx;
    m[11] = 5.0f * (Fy * (ux2 + 3.0f * uy2 + uz2) + 2.0f * uy * (fux + fuz)) - 13.0f * Fy;
    m[12] = 5.0f * (Fz * (ux2 + uy2 + 3.0f * uz2) + 2.0f * uz * (fux + fuy)) - 13.0f * Fz;
    m[13] = Fx * uy * uz + Fy * ux * uz + Fz * ux * uy;
    m[14] = 20.0f * (fux * (3.0f * (uy2 + uz2) - 4.0f) + fuy * (3.0f * (ux2 + uz2) - 4.0f) +
                     fuz * (3.0f * (ux2 + uy2) - 4.0f));
    static_for<15>([&](auto ia) {
        constexpr int a = decltype(ia)::value;
        float s = 0.0f;
        static_for<15>([&](auto ib) {
            constexpr int b = decltype(ib)::value;
            constexpr int k = k15(b, a);
            if constexpr (b >= 1 && k != 0) {
                constexpr float c = float(k) / float(d15(b));
                s = fmaf(c, m[b], s);
            }
        });
        S[a] = s;
    });
}

// The cascade on deviation raw moments.  dk*: raw moments of the deviations
// f - w; returns g[4..14].
__device__ __forceinline__ void kernels15(const float (&f)[15], float Fx, float Fy, float Fz,
                                          const RelaxRates15 &r, float &ux, float &uy, float &uz,
                                          float (&g)[15]) {
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float kxy = 0.f, kxz = 0.f, kyz = 0.f, kxx = 0.f, kyy = 0.f, kzz = 0.f;
    float kxyy = 0.f, kxxy = 0.f, kxxz = 0.f, kxyz = 0.f, kxxyy = 0.f;
    static_for<15>([&](auto ia) {
        constexpr int a = decltype(ia)::value;
        constexpr int x = q15_e(a, 0), y = q15_e(a, 1), z = q15_e(a, 2);
        const float v = f[a];
        drho += v;
        if constexpr (x != 0) {
            jx += x * v;
            kxx += v;
        }
        if constexpr (y != 0) {
            jy += y * v;
            kyy += v;
        }
        if constexpr (z != 0) {
            jz += z * v;
            kzz += v;
        }
        if constexpr (x * y != 0) {
            kxy += (x * y) * v;
            kxyy += x * v;
            kxxy += y * v;
            kxxyy += v;
        }
        if constexpr (x * z != 0) {
            kxz += (x * z) * v;
            kxxz += z * v;
        }
        if constexpr (y * z != 0) kyz += (y * z) * v;
        if constexpr (x * y * z != 0) kxyz += (x * y * z) * v;
    });
    const float rho = 1.0f + drho;
    const float inv_rho = 1.0f / rho;
    ux = (jx + 0.5f * Fx) * inv_rho;
    uy = (jy + 0.5f * Fy) * inv_rho;
    uz = (jz + 0.5f * Fz) * inv_rho;
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    // raw source moments (App. C); eta' = kappa' + sigma' as deviations
    const float sx = Fx, sy = Fy, sz = Fz;
    const float exy = kxy + (Fx * uy + Fy * ux);
    const float exz = kxz + (Fx * uz + Fz * ux);
    const float eyz = kyz + (Fy * uz + Fz * uy);
    const float exx = kxx + 2.0f * Fx * ux;
    const float eyy = kyy + 2.0f * Fy * uy;
    const float ezz = kzz + 2.0f * Fz * uz;
    const float exyy = kxyy + (Fx * uy2 + 2.0f * Fy * uy * ux);
    const float exxy = kxxy + (Fy * ux2 + 2.0f * Fx * ux * uy);
    const float exxz = kxxz + (Fz * ux2 + 2.0f * Fx * ux * uz);
    const float exyz = kxyz + (Fx * uy * uz + Fy * ux * uz + Fz * ux * uy);
    const float exxyy = kxxyy + (2.0f * Fx * ux * uy2 + 2.0f * Fy * uy * ux2);
    const float third = 1.0f / 3.0f;
    const float Exx = third + exx, Eyy = third + eyy;  // full eta'_xx, eta'_yy

#pragma unroll
    for (int b = 0; b < 15; ++b) g[b] = 0.0f;
    g[4] = r.w[4] * 0.125f * (-exy + rho * ux * uy + 0.5f * (sx * uy + sy * ux));
    g[5] = r.w[5] * 0.125f * (-exz + rho * ux * uz + 0.5f * (sx * uz + sz * ux));
    g[6] = r.w[6] * 0.125f * (-eyz + rho * uy * uz + 0.5f * (sy * uz + sz * uy));
    g[7] = r.w[7] * 0.25f * (-(exx - eyy) + rho * (ux2 - uy2) + (sx * ux - sy * uy));
    g[8] = r.w[8] * (1.0f / 12.0f) *
           (-(exx + eyy - 2.0f * ezz) + rho * (ux2 + uy2 - 2.0f * uz2) +
            (sx * ux + sy * uy - 2.0f * sz * uz));
    // -(eta'_xx + eta'_yy + eta'_zz) + rho = -(dev sum) - 1 + rho
    g[9] = r.w[9] * (1.0f / 18.0f) *
           (-(exx + eyy + ezz) + rho * (ux2 + uy2 + uz2) + (sx * ux + sy * uy + sz * uz) + drho);
    g[10] = r.w[10] * 0.0625f *
                (-exyy + 2.0f * uy * exy + ux * Eyy - 2.0f * rho * ux * uy2 - 0.5f * sx * uy2 -
                 sy * uy * ux) +
            uy * g[4] + 0.125f * ux * (-g[7] + g[8] + 3.0f * g[9]);
    g[11] = r.w[11] * 0.0625f *
                (-exxy + 2.0f * ux * exy + uy * Exx - 2.0f * rho * ux2 * uy - 0.5f * sy * ux2 -
                 sx * ux * uy) +
            ux * g[4] + 0.125f * uy * (g[7] + g[8] + 3.0f * g[9]);
    g[12] = r.w[12] * 0.0625f *
                (-exxz + 2.0f * ux * exz + uz * Exx - 2.0f * rho * ux2 * uz - 0.5f * sz * ux2 -
                 sx * ux * uz) +
            ux * g[5] + 0.125f * uz * (g[7] + g[8] + 3.0f * g[9]);
    g[13] = r.w[13] * 0.125f *
                (-exyz + ux * eyz + uy * exz + uz * exy - 2.0f * rho * ux * uy * uz -
                 0.5f * (sx * uy * uz + sy * ux * uz + sz * ux * uy)) +
            uz * g[4] + uy * g[5] + ux * g[6];
    // post-collision kappa~_xx, kappa~_yy as deviations from 1/3
    const float dkx = exx + 2.0f * g[7] + 2.0f * g[8] + 6.0f * g[9] - rho * ux2 - Fx * ux;
    const float dky = eyy - 2.0f * g[7] + 2.0f * g[8] + 6.0f * g[9] - rho * uy2 - Fy * uy;
    // -eta'_xxyy + kappa~_xx kappa~_yy = -dev_xxyy + (dkx + dky)/3 + dkx dky
    g[14] = r.w[14] * 0.0625f *
                (-exxyy + 2.0f * ux * exyy + 2.0f * uy * exxy - ux2 * Eyy - uy2 * Exx -
                 4.0f * ux * uy * exy + (dkx + dky) * third + dkx * dky +
                 3.0f * rho * ux2 * uy2 + sx * ux * uy2 + sy * uy * ux2) -
            2.0f * ux * uy * g[4] + 0.125f * (ux2 - uy2) * g[7] - 0.125f * (ux2 + uy2) * g[8] +
            (-0.375f * (ux2 + uy2) - 0.5f) * g[9] + 2.0f * ux * g[10] + 2.0f * uy * g[11];
}

// One cell: deviations in, post-collision deviations out.
__device__ __forceinline__ void collide15(float (&f)[15], float Fx, float Fy, float Fz,
                                          const RelaxRates15 &r) {
    float g[15], S[15], ux, uy, uz;
    kernels15(f, Fx, Fy, Fz, r, ux, uy, uz, g);
    source15(Fx, Fy, Fz, ux, uy, uz, S);
    static_for<15>([&](auto ia) {
        constexpr int a = decltype(ia)::value;
        float s = f[a] + S[a];
        static_for<15>([&](auto ib) {
            constexpr int b = decltype(ib)::value;
            constexpr int k = k15(b, a);
            if constexpr (b >= 4 && k != 0) s = fmaf(float(k), g[b], s);
        });
        f[a] = s;
    });
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
    RelaxRates15 ones;
#pragma unroll
    for (int b = 0; b < 15; ++b) ones.w[b] = 1.0f;
    float g[15], ux0, uy0, uz0;
    kernels15(f, 0.0f, 0.0f, 0.0f, ones, ux0, uy0, uz0, g);
    float S[15];
    source15(Fx, Fy, Fz, ux, uy, uz, S);
    static_for<15>([&](auto ia) {
        constexpr int a = decltype(ia)::value;
        float s = f[a];
        static_for<15>([&](auto ib) {
            constexpr int b = decltype(ib)::value;
            constexpr int k = k15(b, a);
            if constexpr (b >= 4 && k != 0) s = fmaf(float(k), g[b], s);
        });
        f[a] = s - 0.5f * S[a];
    });
}

}  // namespace lbm
