// Kernels of liblbm.so, templated over the lattice (Q = 27 or 15) and the
// storage type (float, __half, __nv_bfloat16).  kernels_q27.cu and
// kernels_q15.cu instantiate them; api.cu calls the launchers.
#pragma once

#include "collide_q15.cuh"
#include "collide_q27.cuh"
#include "lattice.cuh"

namespace lbm {

struct StepArgs {
    Grid g;
    float w[27];           // relaxation rates omega_beta (first Q used)
    float F[3];            // uniform body force
    const float *Ffield;   // per-cell force [3][nz][ny][nx] or nullptr
};

// Launch geometry shared by the per-cell kernels: blocks of 128 threads laid
// along x (whole warps on a row), several rows per block when nx is short.
struct CellLaunch {
    dim3 grid, block;
};

inline CellLaunch cell_launch(const Grid &g) {
    int bx = ((g.nx + 31) / 32) * 32;
    if (bx > 128) bx = 128;
    int by = 128 / bx;
    if (by < 1) by = 1;
    CellLaunch L;
    L.block = dim3(bx, by, 1);
    L.grid = dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz);
    return L;
}

__device__ __forceinline__ bool cell_coords(const Grid &g, int &x, int &y, int &z) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = blockIdx.z;
    return x < g.nx && y < g.ny;
}

__device__ __forceinline__ long long dense_index(const Grid &g, int x, int y, int z) {
    return ((long long)z * g.ny + y) * g.nx + x;
}

template <int Q>
struct Rates;
template <>
struct Rates<27> {
    using type = RelaxRates27;
};
template <>
struct Rates<15> {
    using type = RelaxRates15;
};

template <int Q>
__device__ __forceinline__ typename Rates<Q>::type load_rates(const StepArgs &a) {
    typename Rates<Q>::type r;
#pragma unroll
    for (int b = 0; b < Q; ++b) r.w[b] = a.w[b];
    return r;
}

template <int Q>
__device__ __forceinline__ void collide(float (&f)[Q], float Fx, float Fy, float Fz,
                                        const typename Rates<Q>::type &r);
template <>
__device__ __forceinline__ void collide<27>(float (&f)[27], float Fx, float Fy, float Fz,
                                            const RelaxRates27 &r) {
    collide27(f, Fx, Fy, Fz, r);
}
template <>
__device__ __forceinline__ void collide<15>(float (&f)[15], float Fx, float Fy, float Fz,
                                            const RelaxRates15 &r) {
    collide15(f, Fx, Fy, Fz, r);
}

template <int Q>
__device__ __forceinline__ void equilibrium(float drho, float ux, float uy, float uz, float Fx,
                                            float Fy, float Fz, float (&f)[Q]);
template <>
__device__ __forceinline__ void equilibrium<27>(float drho, float ux, float uy, float uz,
                                                float Fx, float Fy, float Fz, float (&f)[27]) {
    equilibrium27(drho, ux, uy, uz, Fx, Fy, Fz, f);
}
template <>
__device__ __forceinline__ void equilibrium<15>(float drho, float ux, float uy, float uz,
                                                float Fx, float Fy, float Fz, float (&f)[15]) {
    equilibrium15(drho, ux, uy, uz, Fx, Fy, Fz, f);
}

__device__ __forceinline__ void cell_force(const StepArgs &a, long long c, long long N, float &Fx,
                                           float &Fy, float &Fz) {
    if (a.Ffield) {
        Fx = __ldg(a.Ffield + c);
        Fy = __ldg(a.Ffield + N + c);
        Fz = __ldg(a.Ffield + 2 * N + c);
    } else {
        Fx = a.F[0];
        Fy = a.F[1];
        Fz = a.F[2];
    }
}

// One fused step: pull-gather (streaming with bounce-back), collision, store.
template <int Q, typename T>
__global__ void __launch_bounds__(128) step_kernel(const T *__restrict__ fin,
                                                   T *__restrict__ fout, const StepArgs a) {
    int x, y, z;
    if (!cell_coords(a.g, x, y, z)) return;
    const PullSources s = pull_sources(a.g, x, y, z);
    float f[Q];
    gather<Q, T>(fin, a.g, s, f);
    float Fx, Fy, Fz;
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    cell_force(a, dense_index(a.g, x, y, z), N, Fx, Fy, Fz);
    const typename Rates<Q>::type r = load_rates<Q>(a);
    collide<Q>(f, Fx, Fy, Fz, r);
    store_own<Q, T>(fout, a.g, s.own, f);
}

// Initial state from FP64 density and velocity fields.
template <int Q, typename T>
__global__ void __launch_bounds__(128) init_kernel(T *__restrict__ buf, const StepArgs a,
                                                   const double *__restrict__ rho,
                                                   const double *__restrict__ u) {
    int x, y, z;
    if (!cell_coords(a.g, x, y, z)) return;
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long c = dense_index(a.g, x, y, z);
    float Fx, Fy, Fz;
    cell_force(a, c, N, Fx, Fy, Fz);
    float f[Q];
    equilibrium<Q>(float(rho[c] - 1.0), float(u[c]), float(u[N + c]), float(u[2 * N + c]), Fx, Fy,
                   Fz, f);
    scatter_state<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
}

// Load a dense FP64 state [Q][N] (pre-collision values at their own cells).
template <int Q, typename T>
__global__ void __launch_bounds__(128) set_state_kernel(T *__restrict__ buf, const Grid g,
                                                        const double *__restrict__ fin) {
    int x, y, z;
    if (!cell_coords(g, x, y, z)) return;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long c = dense_index(g, x, y, z);
    float f[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) f[a] = float(fin[a * N + c] - weight<Q>(a));
    scatter_state<Q, T>(buf, g, pull_sources(g, x, y, z), f);
}

// Read the state back as dense FP64 [Q][N].
template <int Q, typename T>
__global__ void __launch_bounds__(128) get_state_kernel(const T *__restrict__ buf, const Grid g,
                                                        double *__restrict__ fout) {
    int x, y, z;
    if (!cell_coords(g, x, y, z)) return;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long c = dense_index(g, x, y, z);
    float f[Q];
    gather<Q, T>(buf, g, pull_sources(g, x, y, z), f);
#pragma unroll
    for (int a = 0; a < Q; ++a) fout[a * N + c] = weight<Q>(a) + double(f[a]);
}

template <int Q>
__device__ __forceinline__ void moments(const float (&f)[Q], float &drho, float &jx, float &jy,
                                        float &jz) {
    drho = jx = jy = jz = 0.0f;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        drho += f[a];
        if (ex<Q>(a)) jx += ex<Q>(a) * f[a];
        if (ey<Q>(a)) jy += ey<Q>(a) * f[a];
        if (ez<Q>(a)) jz += ez<Q>(a) * f[a];
    }
}

// Density and velocity (Eqs. densitycalculation, velocitycalculation).
template <int Q, typename T>
__global__ void __launch_bounds__(128) macro_kernel(const T *__restrict__ buf, const StepArgs a,
                                                    float *__restrict__ rho,
                                                    float *__restrict__ u) {
    int x, y, z;
    if (!cell_coords(a.g, x, y, z)) return;
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long c = dense_index(a.g, x, y, z);
    float f[Q];
    gather<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
    float drho, jx, jy, jz, Fx, Fy, Fz;
    moments<Q>(f, drho, jx, jy, jz);
    cell_force(a, c, N, Fx, Fy, Fz);
    const float r = 1.0f + drho, ir = 1.0f / r;
    if (rho) rho[c] = r;
    if (u) {
        u[c] = (jx + 0.5f * Fx) * ir;
        u[N + c] = (jy + 0.5f * Fy) * ir;
        u[2 * N + c] = (jz + 0.5f * Fz) * ir;
    }
}

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 2048;

// Partial sums of (rho - 1, rho u) per block in FP64, fixed order.
template <int Q, typename T>
__global__ void __launch_bounds__(kRedThreads) conservation_kernel(const T *__restrict__ buf,
                                                                   const StepArgs a,
                                                                   double *__restrict__ part) {
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = int(c % a.g.nx);
        const long long yz = c / a.g.nx;
        const int y = int(yz % a.g.ny), z = int(yz / a.g.ny);
        float f[Q];
        gather<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
        float drho, jx, jy, jz, Fx, Fy, Fz;
        moments<Q>(f, drho, jx, jy, jz);
        cell_force(a, c, N, Fx, Fy, Fz);
        acc[0] += drho;
        acc[1] += double(jx) + 0.5 * Fx;
        acc[2] += double(jy) + 0.5 * Fy;
        acc[3] += double(jz) + 0.5 * Fz;
    }
    __shared__ double sh[4][kRedThreads];
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = sh[k][0];
}

// Launchers.  kernels_q27.cu / kernels_q15.cu hold their explicit
// instantiations; api.cu sees them through the extern declarations below.
template <int Q, typename T>
cudaError_t launch_step(const void *fin, void *fout, const StepArgs &a, cudaStream_t st) {
    const CellLaunch L = cell_launch(a.g);
    step_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<const T *>(fin),
                                                  static_cast<T *>(fout), a);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_init(void *buf, const StepArgs &a, const double *rho, const double *u,
                        cudaStream_t st) {
    const CellLaunch L = cell_launch(a.g);
    init_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<T *>(buf), a, rho, u);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_set_state(void *buf, const Grid &g, const double *f, cudaStream_t st) {
    const CellLaunch L = cell_launch(g);
    set_state_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<T *>(buf), g, f);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_get_state(const void *buf, const Grid &g, double *f, cudaStream_t st) {
    const CellLaunch L = cell_launch(g);
    get_state_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<const T *>(buf), g, f);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_macro(const void *buf, const StepArgs &a, float *rho, float *u,
                         cudaStream_t st) {
    const CellLaunch L = cell_launch(a.g);
    macro_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<const T *>(buf), a, rho, u);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_conservation(const void *buf, const StepArgs &a, double *part, int blocks,
                                cudaStream_t st) {
    conservation_kernel<Q, T><<<blocks, kRedThreads, 0, st>>>(static_cast<const T *>(buf), a,
                                                              part);
    return cudaGetLastError();
}

// Final reduction of the per-block partials to 4 doubles (one block).
cudaError_t launch_reduce_final(const double *part, int blocks, double *out, cudaStream_t st);

// Number of partial-sum blocks the conservation reduction uses for N cells.
inline int conservation_blocks(long long N) {
    long long b = (N + kRedThreads - 1) / kRedThreads;
    if (b > kRedMaxBlocks) b = kRedMaxBlocks;
    if (b < 1) b = 1;
    return int(b);
}

#define LBM_INSTANTIATE_1(EXT, Q, T)                                                             \
    EXT template cudaError_t launch_step<Q, T>(const void *, void *, const StepArgs &,          \
                                               cudaStream_t);                                  \
    EXT template cudaError_t launch_init<Q, T>(void *, const StepArgs &, const double *,         \
                                               const double *, cudaStream_t);                  \
    EXT template cudaError_t launch_set_state<Q, T>(void *, const Grid &, const double *,        \
                                                    cudaStream_t);                             \
    EXT template cudaError_t launch_get_state<Q, T>(const void *, const Grid &, double *,        \
                                                    cudaStream_t);                             \
    EXT template cudaError_t launch_macro<Q, T>(const void *, const StepArgs &, float *, float *, \
                                                cudaStream_t);                                 \
    EXT template cudaError_t launch_conservation<Q, T>(const void *, const StepArgs &, double *, \
                                                       int, cudaStream_t);

#define LBM_INSTANTIATE(EXT, Q)                \
    LBM_INSTANTIATE_1(EXT, Q, float)           \
    LBM_INSTANTIATE_1(EXT, Q, __half)          \
    LBM_INSTANTIATE_1(EXT, Q, __nv_bfloat16)

}  // namespace lbm
