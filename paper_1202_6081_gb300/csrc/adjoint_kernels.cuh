// Kernels of the discrete adjoint of the step (D3Q27 and D3Q15) and of the
// seeds of the objectives (not in the paper: the reverse mode of its update).
//
// Forward step (pull form): f_{t+1}[a](x) = C_a(f_t(x - e_a)), or, behind a
// bounce-back wall, C_opp(a)(f_t(x)).  Its transpose for the adjoint
// lam = dJ/df:
//     lam_t(y) = J_C(f_t(y))^T mu(y),   mu_b(y) = lam_{t+1}[b](y + e_b)
// (or lam_{t+1}[opp b](y) when y + e_b is behind a wall), and
//     dJ/dF(y) += (dC/dF)^T mu(y).
// Adjoint fields are FP32, laid out like the state (population planes of
// pitched rows).
#pragma once

#include "adjoint_q15.cuh"
#include "adjoint_q27.cuh"
#include "kernels.cuh"

namespace lbm {

// Per-cell reverse of the collision, chosen by the lattice (array size).
template <typename V>
__device__ __forceinline__ void adjoint_collide(const V (&f)[27], V Fx, V Fy, V Fz,
                                                const Rates27<V> &r, const V (&mu)[27],
                                                V (&lam)[27], V &gx, V &gy, V &gz) {
    adjoint27<V>(f, Fx, Fy, Fz, r, mu, lam, gx, gy, gz);
}
template <typename V>
__device__ __forceinline__ void adjoint_collide(const V (&f)[15], V Fx, V Fy, V Fz,
                                                const Rates15<V> &r, const V (&mu)[15],
                                                V (&lam)[15], V &gx, V &gy, V &gz) {
    adjoint15<V>(f, Fx, Fy, Fz, r, mu, lam, gx, gy, gz);
}

// The rates of lattice Q in both lanes, from the host-built PackedRates.
template <int Q>
struct PairRates;
template <>
struct PairRates<27> {
    using type = Rates27<f2>;
    static __device__ __forceinline__ type load(const PackedRates &p) {
        return load_rates_packed(p);
    }
};
template <>
struct PairRates<15> {
    using type = Rates15<f2>;
    static __device__ __forceinline__ type load(const PackedRates &p) {
        Rates15<f2> r;
#pragma unroll
        for (int b = 0; b < 15; ++b) r.w[b] = f2(p.w15[b]);
        return r;
    }
};

struct AdjointArgs {
    const float *lam_next[27];  // planes of lam_{t+1} (the first Q used)
    float *lam_out[27];         // planes of lam_t
    float *gF;                  // dense [3][N] accumulator or nullptr
};

template <int Q, typename T, bool kWalls>
__global__ void __launch_bounds__(128) adjoint_kernel(const StepIO<T> io, const AdjointArgs g,
                                                      const StepArgs a) {
    int x, y, z;
    if (!cell_coords(a.g, x, y, z)) return;
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);
    const int xs[3] = {(x + 1 == a.g.nx) ? 0 : x + 1, x, (x == 0) ? a.g.nx - 1 : x - 1};
    float f[Q], mu[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int i = ex<Q>(q) + 1, j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
        // state at t: pull from x - e_q
        const bool wall = kWalls && R.wall[j][k];
        const int src = wall ? R.own + x : R.off[j][k] + xs[i];
        const T *plane = wall ? io.in[opposite<Q>(q)] : io.in[q];
        float v = Storage<T>::load(plane + src);
        if (Storage<T>::kRef && has_ref<Q>(q)) {  // BF16 momentum reference (lattice.cuh)
            const float4 J = __ldg(io.ref_in + (src >> 1));
            const float r = ex<Q>(q) * J.x + ey<Q>(q) * J.y + ez<Q>(q) * J.z;
            v += wall ? -r : r;
        }
        f[q] = Storage<T>::kScaled ? v * float(weight<Q>(q)) : v;
        // adjoint at t+1: from x + e_q (the mirrored pull)
        if (kWalls && R.wall[2 - j][2 - k])
            mu[q] = __ldg(g.lam_next[opposite<Q>(q)] + R.own + x);
        else
            mu[q] = __ldg(g.lam_next[q] + R.off[2 - j][2 - k] + xs[2 - i]);
    }
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long c = dense_index(a.g, x, y, z);
    float Fx, Fy, Fz;
    cell_force(a, c, N, Fx, Fy, Fz);
    const typename Rates<Q>::type r = load_rates<Q>(a);
    float lam[Q], gx, gy, gz;
    adjoint_collide<float>(f, Fx, Fy, Fz, r, mu, lam, gx, gy, gz);
#pragma unroll
    for (int q = 0; q < Q; ++q) __stcs(g.lam_out[q] + R.own + x, lam[q]);
    if (g.gF) {
        g.gF[c] += gx;
        g.gF[N + c] += gy;
        g.gF[2 * N + c] += gz;
    }
}

// The same adjoint step for two neighbouring cells (x0, x0 + 1) per thread in
// packed f32x2 arithmetic (nx even).  The state is pulled as in step2_kernel;
// the adjoint is pulled from the mirrored neighbours x + e_q: for e_x = 0 an
// aligned pair, for e_x = +1 the cells (x0 + 1, x0 + 2), for e_x = -1
// (x0 - 1, x0).
// 3 blocks of 128 threads per SM: 168 registers.  D3Q27 spills a few of its
// 242 there but beats 2 blocks and 4 (128 registers, ~700 B of spills:
// 0.206 vs 0.135 ms at 128^3); D3Q15 fits without spills and beats 4 blocks
// (276 B of spills; 0.098 vs 0.090 ms).
template <int Q, typename T, bool kWalls>
__global__ void __launch_bounds__(128, 3) adjoint2_kernel(const StepIO<T> io, const AdjointArgs g,
                                                       const StepArgs a, const PackedRates pr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    const int x0 = 2 * t;
    if (x0 >= a.g.nx || y >= a.g.ny) return;
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);
    const int xm = (x0 == 0) ? a.g.nx - 1 : x0 - 1;
    const int xp = (x0 + 2 == a.g.nx) ? 0 : x0 + 2;
    const int own = R.own + x0;
    f2 f[Q], mu[Q];
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        constexpr int i = ex<Q>(q), j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
        constexpr int o = opposite<Q>(q);
        f[q] = pull_pair<Q, T, kWalls>(io, R, q, x0, xm, xp);
        if (kWalls && R.wall[2 - j][2 - k]) {
            mu[q] = Pair<float>::ld2(g.lam_next[o] + own);
        } else {
            const float *row = g.lam_next[q] + R.off[2 - j][2 - k];
            if constexpr (i == 0)
                mu[q] = Pair<float>::ld2(row + x0);
            else if constexpr (i == 1)
                mu[q] = f2(__ldg(row + x0 + 1), __ldg(row + xp));
            else
                mu[q] = f2(__ldg(row + xm), __ldg(row + x0));
        }
    });
    // deviations f - w: BF16 references added, 16-bit values scaled by w
    if constexpr (Storage<T>::kRef) add_refs_pair<Q, kWalls>(io.ref_in, R, x0, xm, xp, f);
    if constexpr (Storage<T>::kScaled) {
        static_for<Q>([&](auto iq) {
            constexpr int q = decltype(iq)::value;
            f[q] = f[q] * f2(float(weight<Q>(q)));
        });
    }
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long c = dense_index(a.g, x0, y, z);
    f2 Fx, Fy, Fz;
    if (a.Ffield) {  // 4-byte alignment only is required of the field: single loads
        Fx = f2(__ldg(a.Ffield + c), __ldg(a.Ffield + c + 1));
        Fy = f2(__ldg(a.Ffield + N + c), __ldg(a.Ffield + N + c + 1));
        Fz = f2(__ldg(a.Ffield + 2 * N + c), __ldg(a.Ffield + 2 * N + c + 1));
    } else {
        Fx = f2(a.F[0]);
        Fy = f2(a.F[1]);
        Fz = f2(a.F[2]);
    }
    // the dJ/dF accumulator is read now, so its latency hides behind the
    // collision's reverse; it is written back at the end
    f2 a0 = f2(0.0f), a1 = f2(0.0f), a2 = f2(0.0f);
    if (g.gF) {
        a0 = f2(g.gF[c], g.gF[c + 1]);
        a1 = f2(g.gF[N + c], g.gF[N + c + 1]);
        a2 = f2(g.gF[2 * N + c], g.gF[2 * N + c + 1]);
    }
    const typename PairRates<Q>::type r = PairRates<Q>::load(pr);
    f2 lam[Q], gx, gy, gz;
    adjoint_collide<f2>(f, Fx, Fy, Fz, r, mu, lam, gx, gy, gz);
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        Pair<float>::st2(g.lam_out[q] + own, lam[q]);
    });
    if (g.gF) {
        a0 = a0 + gx;
        a1 = a1 + gy;
        a2 = a2 + gz;
        g.gF[c] = a0.lo();
        g.gF[c + 1] = a0.hi();
        g.gF[N + c] = a1.lo();
        g.gF[N + c + 1] = a1.hi();
        g.gF[2 * N + c] = a2.lo();
        g.gF[2 * N + c + 1] = a2.hi();
    }
}

// Seed of the adjoint for J = sum_x rho |u|^2 / 2 at the final state:
// lam_a = u.e_a - |u|^2 / 2, and the direct term dJ/dF += u / 2
// (u = (j + F/2) / rho).
template <int Q, typename T>
__global__ void __launch_bounds__(128) energy_seed_kernel(const T *__restrict__ buf,
                                                          const StepArgs a, AdjointArgs g) {
    int x, y, z;
    if (!cell_coords(a.g, x, y, z)) return;
    float f[Q];
    gather<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
    float drho, jx, jy, jz, Fx, Fy, Fz;
    moments<Q>(f, drho, jx, jy, jz);
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long c = dense_index(a.g, x, y, z);
    cell_force(a, c, N, Fx, Fy, Fz);
    const float ir = 1.0f / (1.0f + drho);
    const float ux = (jx + 0.5f * Fx) * ir, uy = (jy + 0.5f * Fy) * ir, uz = (jz + 0.5f * Fz) * ir;
    const float h = 0.5f * (ux * ux + uy * uy + uz * uz);
    const long long own = ((long long)z * a.g.ny + y) * a.g.px + x;
#pragma unroll
    for (int q = 0; q < Q; ++q)
        g.lam_out[q][own] = ex<Q>(q) * ux + ey<Q>(q) * uy + ez<Q>(q) * uz - h;
    if (g.gF) {
        g.gF[c] += 0.5f * ux;
        g.gF[N + c] += 0.5f * uy;
        g.gF[2 * N + c] += 0.5f * uz;
    }
}

// Seed of the adjoint for an objective J(rho, u) of the macroscopic fields
// (Eqs. densitycalculation, velocitycalculation) given g_rho = dJ/drho and
// g_u = dJ/du per cell (dense FP32; NULL = zero): since d rho / d f_a = 1 and
// d u_i / d f_a = (e_ai - u_i) / rho,
//     lam_a = g_rho + sum_i (e_ai - u_i) g_u_i / rho,
// and the direct term dJ/dF_i += g_u_i / (2 rho) (u carries F/2).
template <int Q, typename T>
__global__ void __launch_bounds__(128) macro_seed_kernel(const T *__restrict__ buf,
                                                         const StepArgs a, AdjointArgs g,
                                                         const float *__restrict__ g_rho,
                                                         const float *__restrict__ g_u) {
    int x, y, z;
    if (!cell_coords(a.g, x, y, z)) return;
    float f[Q];
    gather<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
    float drho, jx, jy, jz, Fx, Fy, Fz;
    moments<Q>(f, drho, jx, jy, jz);
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long c = dense_index(a.g, x, y, z);
    cell_force(a, c, N, Fx, Fy, Fz);
    const float ir = 1.0f / (1.0f + drho);
    const float ux = (jx + 0.5f * Fx) * ir, uy = (jy + 0.5f * Fy) * ir, uz = (jz + 0.5f * Fz) * ir;
    const float gr = g_rho ? g_rho[c] : 0.0f;
    const float gx = g_u ? g_u[c] * ir : 0.0f;
    const float gy = g_u ? g_u[N + c] * ir : 0.0f;
    const float gz = g_u ? g_u[2 * N + c] * ir : 0.0f;
    const float base = gr - (ux * gx + uy * gy + uz * gz);
    const long long own = ((long long)z * a.g.ny + y) * a.g.px + x;
#pragma unroll
    for (int q = 0; q < Q; ++q)
        g.lam_out[q][own] = base + ex<Q>(q) * gx + ey<Q>(q) * gy + ez<Q>(q) * gz;
    if (g.gF) {
        g.gF[c] += 0.5f * gx;
        g.gF[N + c] += 0.5f * gy;
        g.gF[2 * N + c] += 0.5f * gz;
    }
}

// Per-block partial sums of rho |u|^2 / 2 (slot 0 of each 4-double record),
// rows assigned to blocks as in the conservation reduction.
template <int Q, typename T>
__global__ void __launch_bounds__(kRedThreads) energy_kernel(const T *__restrict__ buf,
                                                             const StepArgs a,
                                                             double *__restrict__ part) {
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long rows = (long long)a.g.ny * a.g.nz;
    double acc = 0.0;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = int(row % a.g.ny), z = int(row / a.g.ny);
        for (int x = threadIdx.x; x < a.g.nx; x += blockDim.x) {
            float f[Q];
            gather<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
            float drho, jx, jy, jz, Fx, Fy, Fz;
            moments<Q>(f, drho, jx, jy, jz);
            cell_force(a, row * a.g.nx + x, N, Fx, Fy, Fz);
            const float px = jx + 0.5f * Fx, py = jy + 0.5f * Fy, pz = jz + 0.5f * Fz;
            acc += double(0.5f * (px * px + py * py + pz * pz) / (1.0f + drho));
        }
    }
    __shared__ double sh[kRedThreads];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[4 * blockIdx.x] = sh[0];
        part[4 * blockIdx.x + 1] = 0.0;
        part[4 * blockIdx.x + 2] = 0.0;
        part[4 * blockIdx.x + 3] = 0.0;
    }
}

template <int Q, typename T>
cudaError_t launch_adjoint(const void *f_t, const float *lam_next, float *lam_out, float *gF,
                           const StepArgs &a, cudaStream_t st) {
    StepIO<T> io{};  // slots q >= Q stay null
    AdjointArgs g{};
    for (int q = 0; q < Q; ++q) {
        io.in[q] = static_cast<const T *>(f_t) + q * a.g.pop;
        io.out[q] = nullptr;
        g.lam_next[q] = lam_next + q * a.g.pop;
        g.lam_out[q] = lam_out + q * a.g.pop;
    }
    io.ref_in = Storage<T>::kRef ? ref_array<Q>(static_cast<const T *>(f_t), a.g.pop, 0) : nullptr;
    g.gF = gF;
    if (a.g.nx % 2 == 0) {
        Grid half = a.g;
        half.nx = a.g.nx / 2;
        const CellLaunch L = cell_launch(half);
        const PackedRates pr = packed_rates(a);
        if (a.g.bc)
            adjoint2_kernel<Q, T, true><<<L.grid, L.block, 0, st>>>(io, g, a, pr);
        else
            adjoint2_kernel<Q, T, false><<<L.grid, L.block, 0, st>>>(io, g, a, pr);
        return cudaGetLastError();
    }
    const CellLaunch L = cell_launch(a.g);
    if (a.g.bc)
        adjoint_kernel<Q, T, true><<<L.grid, L.block, 0, st>>>(io, g, a);
    else
        adjoint_kernel<Q, T, false><<<L.grid, L.block, 0, st>>>(io, g, a);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_energy_seed(const void *f, float *lam_out, float *gF, const StepArgs &a,
                               cudaStream_t st) {
    AdjointArgs g{};
    for (int q = 0; q < Q; ++q) {
        g.lam_next[q] = nullptr;
        g.lam_out[q] = lam_out + q * a.g.pop;
    }
    g.gF = gF;
    const CellLaunch L = cell_launch(a.g);
    energy_seed_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<const T *>(f), a, g);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_macro_seed(const void *f, const float *g_rho, const float *g_u,
                              float *lam_out, float *gF, const StepArgs &a, cudaStream_t st) {
    AdjointArgs g{};
    for (int q = 0; q < Q; ++q) {
        g.lam_next[q] = nullptr;
        g.lam_out[q] = lam_out + q * a.g.pop;
    }
    g.gF = gF;
    const CellLaunch L = cell_launch(a.g);
    macro_seed_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<const T *>(f), a, g, g_rho, g_u);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_energy(const void *f, const StepArgs &a, double *part, int blocks,
                          cudaStream_t st) {
    energy_kernel<Q, T><<<blocks, kRedThreads, 0, st>>>(static_cast<const T *>(f), a, part);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_ADJOINT(EXT, Q, T)                                                        \
    EXT template cudaError_t launch_adjoint<Q, T>(const void *, const float *, float *, float *, \
                                                  const StepArgs &, cudaStream_t);              \
    EXT template cudaError_t launch_energy_seed<Q, T>(const void *, float *, float *,            \
                                                      const StepArgs &, cudaStream_t);          \
    EXT template cudaError_t launch_macro_seed<Q, T>(const void *, const float *, const float *, \
                                                     float *, float *, const StepArgs &,        \
                                                     cudaStream_t);                             \
    EXT template cudaError_t launch_energy<Q, T>(const void *, const StepArgs &, double *, int,  \
                                                 cudaStream_t);

}  // namespace lbm
