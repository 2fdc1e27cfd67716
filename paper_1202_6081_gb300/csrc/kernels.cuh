// Kernels of liblbm.so, templated over the lattice (Q = 27 or 15) and the
// storage type (float, __half, __nv_bfloat16).  kernels_q27_f32.cu,
// kernels_q27_f16.cu, kernels_q27_bf16.cu and kernels_q15.cu instantiate
// them; api.cu calls the launchers.
#pragma once

#include "collide_q15.cuh"
#include "collide_q27.cuh"
#include "lattice.cuh"
#include "vec2.cuh"

#include <cstring>

namespace lbm {

struct StepArgs {
    Grid g;
    float w[27];           // relaxation rates omega_beta (first Q used)
    float F[3];            // uniform body force
    const float *Ffield;   // per-cell force [3][nz][ny][nx] or nullptr
    int has_force;         // 0: no force anywhere (the source term vanishes)
    int sr32;              // FP32 storage: incremental update, stochastically rounded
};

// Launch geometry shared by the per-cell kernels (cell_launch below).
struct CellLaunch {
    dim3 grid, block;
};

// 128-thread blocks along x: rows of at least 17 threads take whole warps
// (32, 64, 96 or 128 threads per row); shorter rows take the next power of
// two, so that a warp covers several rows instead of idling.
inline CellLaunch cell_launch(const Grid &g) {
    int bx;
    if (g.nx <= 16) {
        bx = 1;
        while (bx < g.nx) bx *= 2;
    } else {
        bx = ((g.nx + 31) / 32) * 32;
        if (bx > 128) bx = 128;
    }
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
    using type = Rates27<float>;
};
template <>
struct Rates<15> {
    using type = Rates15<float>;
};

__device__ __forceinline__ Rates27<float> load_rates27(const StepArgs &a) {
    Rates27<float> r;
#pragma unroll
    for (int b = 0; b < 27; ++b) {
        r.w[b] = a.w[b];
        r.nw[b] = -a.w[b];
        r.omw[b] = 1.0f - a.w[b];
    }
    return r;
}

template <int Q>
__device__ __forceinline__ typename Rates<Q>::type load_rates(const StepArgs &a);
template <>
__device__ __forceinline__ Rates27<float> load_rates<27>(const StepArgs &a) {
    return load_rates27(a);
}
template <>
__device__ __forceinline__ Rates15<float> load_rates<15>(const StepArgs &a) {
    Rates15<float> r;
#pragma unroll
    for (int b = 0; b < 15; ++b) r.w[b] = a.w[b] * k15_inv(b);
    return r;
}

template <int Q>
__device__ __forceinline__ void collide(float (&f)[Q], float Fx, float Fy, float Fz,
                                        const typename Rates<Q>::type &r, bool has_force);
template <>
__device__ __forceinline__ void collide<27>(float (&f)[27], float Fx, float Fy, float Fz,
                                            const Rates27<float> &r, bool) {
    collide27<float>(f, Fx, Fy, Fz, r);
}
template <>
__device__ __forceinline__ void collide<15>(float (&f)[15], float Fx, float Fy, float Fz,
                                            const Rates15<float> &r, bool has_force) {
    collide15<float>(f, Fx, Fy, Fz, r, has_force);
}

// The same, returning the cell's velocity (Eq. velocitycalculation).
template <int Q>
__device__ __forceinline__ void collide_u(float (&f)[Q], float Fx, float Fy, float Fz,
                                          const typename Rates<Q>::type &r, bool has_force,
                                          float &ux, float &uy, float &uz);
template <>
__device__ __forceinline__ void collide_u<27>(float (&f)[27], float Fx, float Fy, float Fz,
                                              const Rates27<float> &r, bool, float &ux, float &uy,
                                              float &uz) {
    collide27<float>(f, Fx, Fy, Fz, r, ux, uy, uz);
}
template <>
__device__ __forceinline__ void collide_u<15>(float (&f)[15], float Fx, float Fy, float Fz,
                                              const Rates15<float> &r, bool has_force, float &ux,
                                              float &uy, float &uz) {
    collide15<float>(f, Fx, Fy, Fz, r, has_force, ux, uy, uz);
}

// The change d = f~ - f the collision makes (for the incremental update).
template <int Q>
__device__ __forceinline__ void collide_delta(const float (&f)[Q], float Fx, float Fy, float Fz,
                                              const typename Rates<Q>::type &r, bool has_force,
                                              float (&d)[Q]);
template <>
__device__ __forceinline__ void collide_delta<27>(const float (&f)[27], float Fx, float Fy,
                                                  float Fz, const Rates27<float> &r, bool,
                                                  float (&d)[27]) {
    collide27_delta(f, Fx, Fy, Fz, r, d);
}
template <>
__device__ __forceinline__ void collide_delta<15>(const float (&f)[15], float Fx, float Fy,
                                                  float Fz, const Rates15<float> &r,
                                                  bool has_force, float (&d)[15]) {
    collide15_delta(f, Fx, Fy, Fz, r, has_force, d);
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

// Base pointer of every population plane of the source and destination
// buffers (plane alpha starts at buf + alpha * pop).  Passed by value, the
// table sits in the constant bank, so each access is one multiply-add of a
// 32-bit element offset onto a constant-bank base.
template <typename T>
struct StepIO {
    const T *in[27];
    T *out[27];
    const float4 *ref_in;  // momentum references of the input state (BF16), else unused
    float4 *ref_out;       // and of the output state
};

// 2-cell pair helpers for the packed kernel (x0 even, row pitch even).
template <typename T>
struct Pair;
// State loads: read-only, with an L2 prefetch-size hint of 256 bytes (the
// pulls stream through whole rows; measured +2.4 % FP16, +1.5 % BF16 at
// 512^3, FP32 unchanged).
__device__ __forceinline__ unsigned long long ld_nc_256_b64(const void *p) {
    unsigned long long v;
    asm("ld.global.nc.L2::256B.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned ld_nc_256_b32(const void *p) {
    unsigned v;
    asm("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned short ld_nc_256_b16(const void *p) {
    unsigned short v;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
template <>
struct Pair<float> {
    __device__ __forceinline__ static f2 ld2(const float *p) { return f2(ld_nc_256_b64(p)); }
    __device__ __forceinline__ static float ld1(const float *p) {
        return __uint_as_float(ld_nc_256_b32(p));
    }
    __device__ __forceinline__ static void st2(float *p, f2 v) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(v.lo(), v.hi()));
    }
    // the step's stores (plain stores for FP32; see Pair16 for 16-bit)
    template <int q>
    __device__ __forceinline__ static void st2s(float *p, f2 v, unsigned) {
        st2(p, v);
    }
    template <int q>
    __device__ __forceinline__ static void st1x2s(float *plo, float *phi, f2 v, unsigned) {
        __stcs(plo, v.lo());
        __stcs(phi, v.hi());
    }
};
// 16-bit step stores: the pair is rounded together (pack_sr) and stored as one
// 32-bit word, or as two halves at separate addresses.
template <typename T>
struct Pair16 {
    template <int q>
    __device__ __forceinline__ static void st2s(T *p, f2 v, unsigned seed) {
        __stcs(reinterpret_cast<unsigned int *>(p), pack_sr<T, q>(v.lo(), v.hi(), seed));
    }
    template <int q>
    __device__ __forceinline__ static void st1x2s(T *plo, T *phi, f2 v, unsigned seed) {
        const unsigned d = pack_sr<T, q>(v.lo(), v.hi(), seed);
        __stcs(reinterpret_cast<unsigned short *>(plo), static_cast<unsigned short>(d & 0xffffu));
        __stcs(reinterpret_cast<unsigned short *>(phi), static_cast<unsigned short>(d >> 16));
    }
};
template <>
struct Pair<__half> : Pair16<__half> {
    __device__ __forceinline__ static f2 ld2(const __half *p) {
        const unsigned w = ld_nc_256_b32(p);
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        return f2(v.x, v.y);
    }
    __device__ __forceinline__ static float ld1(const __half *p) {
        return __half2float(__ushort_as_half(ld_nc_256_b16(p)));
    }
};
template <>
struct Pair<__nv_bfloat16> : Pair16<__nv_bfloat16> {
    __device__ __forceinline__ static f2 ld2(const __nv_bfloat16 *p) {
        const unsigned w = ld_nc_256_b32(p);
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
        return f2(v.x, v.y);
    }
    __device__ __forceinline__ static float ld1(const __nv_bfloat16 *p) {
        return __bfloat162float(__ushort_as_bfloat16(ld_nc_256_b16(p)));
    }
};

// Seed of a thread's stochastic rounding (sr_seed) from four of its
// pre-collision values, of different directions, and its position.
template <int Q>
constexpr int kSeedPop = Q == 27 ? 11 : 9;
template <int Q>
__device__ __forceinline__ unsigned pair_seed(const f2 (&f)[Q], int own) {
    return sr_seed(f[1].v ^ f[6].v ^ f[kSeedPop<Q>].v ^ f[Q - 1].v, own);
}
// Which values the pair kernels hash: the pre-collision ones, or for D3Q15
// with FP16 storage the post-collision ones (either is a fixed function of
// the state; chosen by measurement: D3Q15 FP16 68.0k vs 62.4k MLUPS at 256^3
// hashing after the collision, D3Q15 BF16 61.5k vs 64.0k and D3Q27 the same
// or better before it).  The in-place kernels make the same choice, so that
// their states stay bit-identical to the two-buffer step's.
template <int Q, typename T>
constexpr bool kSeedAfterCollision = Q == 15 && Storage<T>::kScaled && !Storage<T>::kRef;

template <int Q>
__device__ __forceinline__ unsigned cell_seed(const float (&f)[Q], int own) {
    const unsigned a = __float_as_uint(f[1]) ^ __float_as_uint(f[6]);
    const unsigned b = __float_as_uint(f[kSeedPop<Q>]) ^ __float_as_uint(f[Q - 1]);
    return sr_seed(static_cast<unsigned long long>(b) << 32 | a, own);
}

// Relaxation rates pre-broadcast to both lanes, built on the host:
// D3Q27 omega, -omega, 1 - omega (divided by 216 for the kernels that fold
// the weights of 16-bit storage into their sums); D3Q15 omega / k_beta.
struct PackedRates {
    unsigned long long w[27], nw[27], omw[27];
    unsigned long long w15[15];
};

__device__ __forceinline__ Rates27<f2> load_rates_packed(const PackedRates &p) {
    Rates27<f2> r;
#pragma unroll
    for (int b = 0; b < 27; ++b) {
        r.w[b] = f2(p.w[b]);
        r.nw[b] = f2(p.nw[b]);
        r.omw[b] = f2(p.omw[b]);
    }
    return r;
}

// Factors of the two-cell kernels between stored values and the collision's
// values.  D3Q27 uses collide27_g: 16-bit inputs go in as stored (the
// weights are folded into its sums), and outputs carry G_i G_j G_k.
template <int Q, typename T>
__host__ __device__ constexpr bool kFoldedLoad() {
    return Q == 27 && Storage<T>::kScaled;
}
template <int Q, typename T>
__host__ __device__ constexpr float load_scale(int q) {
    return (Storage<T>::kScaled && Q != 27) ? float(weight<Q>(q)) : 1.0f;
}
template <int Q, typename T>
__host__ __device__ constexpr float store_scale(int q) {
    return float((Storage<T>::kScaled ? 1.0 / weight<Q>(q) : 1.0) / (Q == 27 ? g27(q) : 1));
}

// Row offsets (elements) of the 3 x 3 source rows of a pull, for cell row
// (y, z); wall[j][k] set where that source is beyond a bounce-back wall.
template <bool kWalls>
struct Rows {
    int off[3][3];
    bool wall[3][3];
    int own;
};

template <bool kWalls>
__device__ __forceinline__ Rows<kWalls> pull_rows(const Grid &g, int y, int z) {
    Rows<kWalls> r;
    const int ys[3] = {(y + 1 == g.ny) ? 0 : y + 1, y, (y == 0) ? g.ny - 1 : y - 1};
    const int zs[3] = {(z + 1 == g.nz) ? 0 : z + 1, z, (z == 0) ? g.nz - 1 : z - 1};
    bool wy[3] = {false, false, false}, wz[3] = {false, false, false};
    if (kWalls) {
        wy[0] = (y + 1 == g.ny) && (g.bc & kWallY);
        wy[2] = (y == 0) && (g.bc & kWallY);
        wz[0] = (z + 1 == g.nz) && (g.bc & kWallZ);
        wz[2] = (z == 0) && (g.bc & kWallZ);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            r.off[j][k] = (zs[k] * g.ny + ys[j]) * g.px;
            r.wall[j][k] = kWalls && (wy[j] || wz[k]);
        }
    r.own = (z * g.ny + y) * g.px;
    return r;
}

// BF16 momentum references (see lattice.cuh) for the pair kernels.
//
// Reader: adds to the pulled raw values f[q] of cells (x0, x0 + 1) the
// reference of each value's producer: for e_x = 0 both from the pair of the
// source row, for e_x = +1 from the pairs of x0 - 1 and x0, for e_x = -1 of
// x0 + 1 and x0 + 2; behind a wall minus that of the own pair.  A source row
// (e_y, e_z) needs two components of J at most, loaded narrow to keep
// registers free: the row e_y = e_z = 0 only Jx (axis populations), rows
// with e_z = 0 (Jx, Jy), rows with e_y = 0 (Jz, Jx) -- J is stored as
// (Jx, Jy, Jz, Jx) so that both pairs are aligned 8-byte loads -- and the
// rows with e_y, e_z both nonzero (Jy, Jz), only of the own column (their
// corners carry no reference).
template <int ey, int ez>
__device__ __forceinline__ float4 load_ref(const float4 *p) {
    if constexpr (ey == 0 && ez == 0) {
        return make_float4(__ldg(&p->x), 0.0f, 0.0f, 0.0f);
    } else if constexpr (ez == 0) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        return make_float4(v.x, v.y, 0.0f, 0.0f);
    } else if constexpr (ey == 0) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p) + 1);
        return make_float4(v.y, 0.0f, v.x, 0.0f);
    } else {
        return __ldg(p);
    }
}

template <int Q, bool kWalls>
__device__ __forceinline__ void add_refs_pair(const float4 *__restrict__ ref, const Rows<kWalls> &R,
                                              int x0, int xm, int xp, f2 (&f)[Q]) {
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        if constexpr (has_ref<Q>(q)) {
            constexpr int i = ex<Q>(q), j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
            constexpr int cy = ey<Q>(q), cz = ez<Q>(q);
            float rlo, rhi;
            if (kWalls && R.wall[j][k]) {
                rlo = rhi = -ref_dot<Q, q>(load_ref<cy, cz>(ref + ((R.own + x0) >> 1)));
            } else {
                const float4 *row = ref + (R.off[j][k] >> 1);
                const float4 C = load_ref<cy, cz>(row + (x0 >> 1));
                if constexpr (i == 0) {
                    rlo = rhi = ref_dot<Q, q>(C);
                } else if constexpr (i == 1) {
                    rlo = ref_dot<Q, q>(load_ref<cy, cz>(row + (xm >> 1)));
                    rhi = ref_dot<Q, q>(C);
                } else {
                    rlo = ref_dot<Q, q>(C);
                    rhi = ref_dot<Q, q>(load_ref<cy, cz>(row + (xp >> 1)));
                }
            }
            f[q] = f[q] + f2(rlo, rhi);
        }
    });
}

// Writer: the pair's reference J = 3 u-bar (mean velocity of the two cells).
__device__ __forceinline__ float4 pair_ref(f2 ux, f2 uy, f2 uz) {
    const float jx = 1.5f * (ux.lo() + ux.hi());
    return make_float4(jx, 1.5f * (uy.lo() + uy.hi()), 1.5f * (uz.lo() + uz.hi()), jx);
}

// Stored value of population q of a pair from its post-collision value v
// times the store scale sc: v sc, minus e_q . J for the referenced
// populations of BF16 storage.
template <int Q, typename T, int q>
__device__ __forceinline__ f2 stored_pair(f2 v, float sc, const float4 &J) {
    if constexpr (Storage<T>::kRef && has_ref<Q>(q))
        return vfma(v, f2(sc), f2(-ref_dot<Q, q>(J)));
    else
        return sc == 1.0f ? v : v * f2(sc);
}

// One fused step, one cell per thread: pull-gather (streaming with
// bounce-back), collision, store.  With BF16 momentum references the cells
// x (even) and x + 1, held by neighbouring lanes, exchange their velocities
// for the pair's reference, so every lane takes part: cells beyond the grid
// edge compute on a clamped cell and store nothing.
// kSR (FP32 storage, opt-in): the update is f~ = f + d with d the
// collision's change, and that last addition is rounded stochastically
// (add_sr32), so that no rounding error repeats identically step after step
// at a steady state.
template <int Q, typename T, bool kWalls, bool kSR = false>
__global__ void __launch_bounds__(128) step_kernel(const StepIO<T> io, const StepArgs a) {
    int x, y, z;
    const bool inside = cell_coords(a.g, x, y, z);
    if constexpr (Storage<T>::kRef) {
        x = min(x, a.g.nx - 1);
        y = min(y, a.g.ny - 1);
    } else {
        if (!inside) return;
    }
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);
    const int xs[3] = {(x + 1 == a.g.nx) ? 0 : x + 1, x, (x == 0) ? a.g.nx - 1 : x - 1};
    float f[Q];
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        constexpr int i = ex<Q>(q) + 1, j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
        const bool wall = kWalls && R.wall[j][k];
        const int src = wall ? R.own + x : R.off[j][k] + xs[i];
        const T *plane = wall ? io.in[opposite<Q>(q)] : io.in[q];
        float v = Storage<T>::load(plane + src);
        if constexpr (Storage<T>::kRef && has_ref<Q>(q)) {
            const float r = ref_dot<Q, q>(__ldg(io.ref_in + (src >> 1)));
            v += wall ? -r : r;
        }
        f[q] = Storage<T>::kScaled ? v * float(weight<Q>(q)) : v;
    });
    const unsigned seed = cell_seed<Q>(f, R.own + x);
    float Fx, Fy, Fz;
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    cell_force(a, dense_index(a.g, x, y, z), N, Fx, Fy, Fz);
    const typename Rates<Q>::type r = load_rates<Q>(a);
    float ux, uy, uz;
    if constexpr (kSR) {
        float d[Q];
        collide_delta<Q>(f, Fx, Fy, Fz, r, a.has_force != 0, d);
        static_for<Q>([&](auto iq) {
            constexpr int q = decltype(iq)::value;
            f[q] = add_sr32(f[q], d[q], sr_bits<q>(seed));
        });
    } else {
        collide_u<Q>(f, Fx, Fy, Fz, r, a.has_force != 0, ux, uy, uz);
    }
    float4 J = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if constexpr (Storage<T>::kRef) {
        const float px = __shfl_xor_sync(0xffffffffu, ux, 1);
        const float py = __shfl_xor_sync(0xffffffffu, uy, 1);
        const float pz = __shfl_xor_sync(0xffffffffu, uz, 1);
        if ((x ^ 1) < a.g.nx)  // both cells of the pair exist (a + b == b + a exactly)
            J = make_float4(1.5f * (ux + px), 1.5f * (uy + py), 1.5f * (uz + pz), 0.0f);
        else
            J = make_float4(3.0f * ux, 3.0f * uy, 3.0f * uz, 0.0f);
        J.w = J.x;
        if (!inside) return;
        if ((x & 1) == 0) __stcs(io.ref_out + ((R.own + x) >> 1), J);
    }
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        float ref = 0.0f;
        if constexpr (Storage<T>::kRef && has_ref<Q>(q)) ref = ref_dot<Q, q>(J);
        store_dev_step<Q, T, q>(io.out[q] + R.own + x, f[q], seed, ref);
    });
}

// One fused D3Q27 step, two neighbouring cells (x0, x0 + 1) per thread with
// the collision in packed f32x2 arithmetic.  nx must be even.  Loads of
// populations with e_x = 0 and all stores are aligned 2-element accesses;
// e_x = +-1 sources are two single loads (x0 - 1, x0) or (x0 + 1, x0 + 2).
// Blocks of 128 per SM, by measurement: FP32 storage 5 (96 registers, no
// spills; 6 blocks ran the same, 32.20k vs 32.23k MLUPS at 256^3, and 7
// slower); 16-bit storage 6 (80 registers): with the rate-1 relaxation FP16
// 48.2k / 48.0k MLUPS at 6 / 7 blocks at 512^3 (before it 41.2k / 44.3k /
// 37.5k at 5 / 6 / 7), BF16 with its reference loads 38.6k / 39.4k at 5 / 6.
template <typename T>
constexpr int kStep2Blocks = Storage<T>::kScaled ? 6 : 5;

// kEq: the rates from the trace on are all 1 (relax27).
template <typename T, bool kWalls, bool kEq>
__global__ void __launch_bounds__(128, kStep2Blocks<T>) step2_kernel(const StepIO<T> io,
                                                                  const StepArgs a,
                                                                  const PackedRates pr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    const int x0 = 2 * t;
    if (x0 >= a.g.nx || y >= a.g.ny) return;
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);
    const int xm = (x0 == 0) ? a.g.nx - 1 : x0 - 1;
    const int xp = (x0 + 2 == a.g.nx) ? 0 : x0 + 2;
    f2 f[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        const int i = ex<27>(q), j = ey<27>(q) + 1, k = ez<27>(q) + 1;
        f2 v;
        if (kWalls && R.wall[j][k]) {
            v = Pair<T>::ld2(io.in[opposite<27>(q)] + R.own + x0);
        } else {
            const T *row = io.in[q] + R.off[j][k];
            if (i == 0)
                v = Pair<T>::ld2(row + x0);
            else if (i == 1)
                v = f2(Pair<T>::ld1(row + xm), Pair<T>::ld1(row + x0));
            else
                v = f2(Pair<T>::ld1(row + x0 + 1), Pair<T>::ld1(row + xp));
        }
        f[q] = v;  // weight-scaled 16-bit values go in as stored (collide27_g)
    }
    if constexpr (Storage<T>::kRef) add_refs_pair<27, kWalls>(io.ref_in, R, x0, xm, xp, f);
    const unsigned seed = pair_seed<27>(f, R.own + x0);
    f2 Fx, Fy, Fz;
    if (a.Ffield) {
        const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
        const long long c = dense_index(a.g, x0, y, z);
        Fx = f2(__ldg(a.Ffield + c), __ldg(a.Ffield + c + 1));
        Fy = f2(__ldg(a.Ffield + N + c), __ldg(a.Ffield + N + c + 1));
        Fz = f2(__ldg(a.Ffield + 2 * N + c), __ldg(a.Ffield + 2 * N + c + 1));
    } else {
        Fx = f2(a.F[0]);
        Fy = f2(a.F[1]);
        Fz = f2(a.F[2]);
    }
    const Rates27<f2> r = load_rates_packed(pr);
    f2 ux, uy, uz;
    collide27_g<f2, Storage<T>::kScaled, kEq>(f, Fx, Fy, Fz, r, ux, uy, uz);
    float4 J = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if constexpr (Storage<T>::kRef) {
        J = pair_ref(ux, uy, uz);
        __stcs(io.ref_out + ((R.own + x0) >> 1), J);
    }
    static_for<27>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        const f2 v = stored_pair<27, T, q>(f[q], store_scale<27, T>(q), J);
        Pair<T>::template st2s<q>(io.out[q] + R.own + x0, v, seed);
    });
}

// Pair gather for lattice Q: population q of cells (x0, x0 + 1) from the pull
// sources (see step2_kernel).
template <int Q, typename T, bool kWalls>
__device__ __forceinline__ f2 pull_pair(const StepIO<T> &io, const Rows<kWalls> &R, int q, int x0,
                                        int xm, int xp) {
    const int i = ex<Q>(q), j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
    if (kWalls && R.wall[j][k]) return Pair<T>::ld2(io.in[opposite<Q>(q)] + R.own + x0);
    const T *row = io.in[q] + R.off[j][k];
    if (i == 0) return Pair<T>::ld2(row + x0);
    if (i == 1) return f2(Pair<T>::ld1(row + xm), Pair<T>::ld1(row + x0));
    return f2(Pair<T>::ld1(row + x0 + 1), Pair<T>::ld1(row + xp));
}

// Body force of the pair (x0, x0 + 1): the field, else the uniform force.
__device__ __forceinline__ void pair_force(const StepArgs &a, int x0, int y, int z, f2 &Fx, f2 &Fy,
                                           f2 &Fz) {
    if (a.Ffield) {
        const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
        const long long c = dense_index(a.g, x0, y, z);
        Fx = f2(__ldg(a.Ffield + c), __ldg(a.Ffield + c + 1));
        Fy = f2(__ldg(a.Ffield + N + c), __ldg(a.Ffield + N + c + 1));
        Fz = f2(__ldg(a.Ffield + 2 * N + c), __ldg(a.Ffield + 2 * N + c + 1));
    } else {
        Fx = f2(a.F[0]);
        Fy = f2(a.F[1]);
        Fz = f2(a.F[2]);
    }
}

// One fused D3Q15 step, two neighbouring cells per thread in packed f32x2
// arithmetic (nx even); loads and stores as in step2_kernel.
// kForce = false (no force anywhere) compiles the force-free cascade alone:
// without the forced path beside it the kernel needs fewer registers (no
// spills at 5 blocks per SM with 16-bit storage, against 104-128 bytes;
// FP16 77.2k against 70.7k MLUPS at 256^3).  Blocks per SM with 16-bit
// storage, from measurement: 6 without force (32-56 bytes of spills; FP16
// 79.2k MLUPS, 78.2k at 7), 5 with it; FP32 storage 4 (no spills; without
// force its 94 registers admit 5).
template <typename T, bool kForce>
constexpr int kQ15Blocks = Storage<T>::kScaled ? (kForce ? 5 : 6) : 4;

template <typename T, bool kWalls, bool kForce>
__global__ void __launch_bounds__(128, (kQ15Blocks<T, kForce>))
    step2_q15_kernel(const StepIO<T> io, const StepArgs a, const PackedRates pr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    const int x0 = 2 * t;
    if (x0 >= a.g.nx || y >= a.g.ny) return;
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);
    const int xm = (x0 == 0) ? a.g.nx - 1 : x0 - 1;
    const int xp = (x0 + 2 == a.g.nx) ? 0 : x0 + 2;
    f2 f[15];
    static_for<15>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        f[q] = pull_pair<15, T, kWalls>(io, R, q, x0, xm, xp);
    });
    if constexpr (Storage<T>::kRef) add_refs_pair<15, kWalls>(io.ref_in, R, x0, xm, xp, f);
    if constexpr (Storage<T>::kScaled) {
        static_for<15>([&](auto iq) {
            constexpr int q = decltype(iq)::value;
            f[q] = f[q] * f2(float(weight<15>(q)));
        });
    }
    unsigned seed = 0;
    if constexpr (!kSeedAfterCollision<15, T>) seed = pair_seed<15>(f, R.own + x0);
    f2 Fx = f2(0.0f), Fy = f2(0.0f), Fz = f2(0.0f);
    if constexpr (kForce) pair_force(a, x0, y, z, Fx, Fy, Fz);
    Rates15<f2> r;
#pragma unroll
    for (int b = 0; b < 15; ++b) r.w[b] = f2(pr.w15[b]);
    f2 ux, uy, uz;
    collide15<f2>(f, Fx, Fy, Fz, r, kForce, ux, uy, uz);
    float4 J = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if constexpr (Storage<T>::kRef) {
        J = pair_ref(ux, uy, uz);
        __stcs(io.ref_out + ((R.own + x0) >> 1), J);
    }
    if constexpr (kSeedAfterCollision<15, T>) seed = pair_seed<15>(f, R.own + x0);
    static_for<15>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        const f2 v = stored_pair<15, T, q>(f[q], store_scale<15, T>(q), J);
        Pair<T>::template st2s<q>(io.out[q] + R.own + x0, v, seed);
    });
}

// ---- in-place (AA) streaming: one buffer, two kinds of step -------------
//
// Even step (layout kAANatural -> kAASwapped): each cell reads its own
// populations f_a(x) from slot a, collides, and writes f~_a(x) back to its
// own cell, slot opp(a).  Odd step (kAASwapped -> kAANatural): each cell
// reads f_a(x) = f~_a(x - e_a) from slot opp(a) of its upstream neighbour (or
// from its own slot a behind a bounce-back wall), collides, and writes
// f~_a(x) to slot a of its downstream neighbour x + e_a (or to its own slot
// opp(a) when x + e_a is behind a wall), where the next even step reads it.
// In both steps a thread reads and writes the same set of locations, so the
// update is race-free in place.  Both use two cells per thread (nx even).

template <int Q>
struct PairCollide;
// kForce = false: no force anywhere (D3Q15 then takes the force-free
// cascade; the D3Q27 collision takes any force, zero included, the same way).
template <>
struct PairCollide<27> {
    template <bool kWeighted, bool kEq, bool>
    __device__ __forceinline__ static void run(f2 (&f)[27], f2 Fx, f2 Fy, f2 Fz,
                                               const PackedRates &pr, f2 &ux, f2 &uy, f2 &uz) {
        const Rates27<f2> r = load_rates_packed(pr);
        collide27_g<f2, kWeighted, kEq>(f, Fx, Fy, Fz, r, ux, uy, uz);
    }
};
template <>
struct PairCollide<15> {
    template <bool, bool, bool kForce>
    __device__ __forceinline__ static void run(f2 (&f)[15], f2 Fx, f2 Fy, f2 Fz,
                                               const PackedRates &pr, f2 &ux, f2 &uy, f2 &uz) {
        Rates15<f2> r;
#pragma unroll
        for (int b = 0; b < 15; ++b) r.w[b] = f2(pr.w15[b]);
        collide15<f2>(f, Fx, Fy, Fz, r, kForce, ux, uy, uz);
    }
};

// Raw pulled values -> the collision's inputs: BF16 references added (their
// producers are the pull sources, see lattice.cuh), then the load scale.
template <int Q, typename T, bool kWalls>
__device__ __forceinline__ void pair_inputs(const StepIO<T> &io, const Rows<kWalls> &R, int x0,
                                            int xm, int xp, f2 (&f)[Q]) {
    if constexpr (Storage<T>::kRef) add_refs_pair<Q, kWalls>(io.ref_in, R, x0, xm, xp, f);
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        constexpr float sc = load_scale<Q, T>(q);
        if constexpr (sc != 1.0f) f[q] = f[q] * f2(sc);
    });
}

// The collision of an in-place step, then the pair's reference (BF16).
template <int Q, typename T, bool kEq, bool kForce>
__device__ __forceinline__ float4 pair_collide(const StepIO<T> &io, const StepArgs &a,
                                               const PackedRates &pr, int x0, int y, int z,
                                               int own, f2 (&f)[Q]) {
    f2 Fx = f2(0.0f), Fy = f2(0.0f), Fz = f2(0.0f), ux, uy, uz;
    if constexpr (kForce) pair_force(a, x0, y, z, Fx, Fy, Fz);
    PairCollide<Q>::template run<kFoldedLoad<Q, T>(), kEq, kForce>(f, Fx, Fy, Fz, pr, ux, uy, uz);
    float4 J = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if constexpr (Storage<T>::kRef) {
        J = pair_ref(ux, uy, uz);
        __stcs(io.ref_out + (own >> 1), J);
    }
    return J;
}

template <int Q, typename T, bool kWalls, bool kEq, bool kForce>
__global__ void __launch_bounds__(128) aa_even_kernel(const StepIO<T> io, const StepArgs a,
                                                      const PackedRates pr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    const int x0 = 2 * t;
    if (x0 >= a.g.nx || y >= a.g.ny) return;
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);  // producers of the values (BF16)
    const int xm = (x0 == 0) ? a.g.nx - 1 : x0 - 1;
    const int xp = (x0 + 2 == a.g.nx) ? 0 : x0 + 2;
    const int own = R.own + x0;
    f2 f[Q];
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        f[q] = Pair<T>::ld2(io.in[q] + own);
    });
    pair_inputs<Q, T, kWalls>(io, R, x0, xm, xp, f);
    unsigned seed = 0;
    if constexpr (!kSeedAfterCollision<Q, T>) seed = pair_seed<Q>(f, own);
    const float4 J = pair_collide<Q, T, kEq, kForce>(io, a, pr, x0, y, z, own, f);
    if constexpr (kSeedAfterCollision<Q, T>) seed = pair_seed<Q>(f, own);
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        const f2 v = stored_pair<Q, T, q>(f[q], store_scale<Q, T>(q), J);
        Pair<T>::template st2s<q>(io.out[opposite<Q>(q)] + own, v, seed);
    });
}

// Blocks of 128 per SM, from measurement: D3Q27 at 5 (96 registers; FP32
// storage without spills, 16-bit with 40 bytes: 38.3k vs 33.3k MLUPS FP16 at
// 512^3 against 3 blocks); D3Q15 with force at 4 (8-48 bytes of spills),
// without force at 5 (no spills; FP16 77.7k vs 68.9k MLUPS at 256^3 against 4).
template <int Q, typename T, bool kForce>
constexpr int kAAOddBlocks = Q == 27 ? 5 : (kForce ? 4 : 5);

template <int Q, typename T, bool kWalls, bool kEq, bool kForce>
__global__ void __launch_bounds__(128, (kAAOddBlocks<Q, T, kForce>))
    aa_odd_kernel(const StepIO<T> io, const StepArgs a, const PackedRates pr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    const int x0 = 2 * t;
    if (x0 >= a.g.nx || y >= a.g.ny) return;
    const Rows<kWalls> R = pull_rows<kWalls>(a.g, y, z);
    const int xm = (x0 == 0) ? a.g.nx - 1 : x0 - 1;
    const int xp = (x0 + 2 == a.g.nx) ? 0 : x0 + 2;
    const int own = R.own + x0;
    f2 f[Q];
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        constexpr int i = ex<Q>(q), j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
        constexpr int o = opposite<Q>(q);
        f2 v;
        if (kWalls && R.wall[j][k]) {
            v = Pair<T>::ld2(io.in[q] + own);
        } else {
            const T *row = io.in[o] + R.off[j][k];
            if constexpr (i == 0)
                v = Pair<T>::ld2(row + x0);
            else if constexpr (i == 1)
                v = f2(Pair<T>::ld1(row + xm), Pair<T>::ld1(row + x0));
            else
                v = f2(Pair<T>::ld1(row + x0 + 1), Pair<T>::ld1(row + xp));
        }
        f[q] = v;
    });
    pair_inputs<Q, T, kWalls>(io, R, x0, xm, xp, f);
    unsigned seed = 0;
    if constexpr (!kSeedAfterCollision<Q, T>) seed = pair_seed<Q>(f, own);
    const float4 J = pair_collide<Q, T, kEq, kForce>(io, a, pr, x0, y, z, own, f);
    if constexpr (kSeedAfterCollision<Q, T>) seed = pair_seed<Q>(f, own);
    static_for<Q>([&](auto iq) {
        constexpr int q = decltype(iq)::value;
        constexpr int i = ex<Q>(q), j = ey<Q>(q) + 1, k = ez<Q>(q) + 1;
        constexpr int o = opposite<Q>(q);
        const f2 v = stored_pair<Q, T, q>(f[q], store_scale<Q, T>(q), J);
        // downstream neighbour x + e_q: the row of the mirrored pull
        if (kWalls && R.wall[2 - j][2 - k]) {
            Pair<T>::template st2s<q>(io.out[o] + own, v, seed);
        } else {
            T *row = io.out[q] + R.off[2 - j][2 - k];
            if constexpr (i == 0)
                Pair<T>::template st2s<q>(row + x0, v, seed);
            else if constexpr (i == 1)
                Pair<T>::template st1x2s<q>(row + x0 + 1, row + xp, v, seed);
            else
                Pair<T>::template st1x2s<q>(row + xm, row + x0, v, seed);
        }
    });
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

// BF16 momentum references of a state being loaded (reference array 0), one
// thread per pair of cells: J = 3 x the mean velocity of the pair, from the
// velocity field u when given, else from the momentum of the distributions
// f (dense FP64 [Q][N]).  Any J would do as long as the values are stored
// and read against the same one; this one keeps the stored values small.
template <int Q, typename T>
__global__ void __launch_bounds__(128) ref_init_kernel(T *__restrict__ buf, const Grid g,
                                                       const double *__restrict__ u,
                                                       const double *__restrict__ f) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    const int x0 = 2 * t;
    if (x0 >= g.nx || y >= g.ny) return;
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long c = dense_index(g, x0, y, z);
    const int n = (x0 + 1 < g.nx) ? 2 : 1;
    float v[2][3];
    for (int m = 0; m < n; ++m)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double sum = 0.0;
            if (u) {
                sum = u[d * N + c + m];
            } else {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int e = d == 0 ? ex<Q>(q) : d == 1 ? ey<Q>(q) : ez<Q>(q);
                    if (e) sum += e * f[q * N + c + m];
                }
            }
            v[m][d] = float(sum);
        }
    float4 J = n == 2 ? make_float4(1.5f * (v[0][0] + v[1][0]), 1.5f * (v[0][1] + v[1][1]),
                                    1.5f * (v[0][2] + v[1][2]), 0.0f)
                      : make_float4(3.0f * v[0][0], 3.0f * v[0][1], 3.0f * v[0][2], 0.0f);
    J.w = J.x;  // stored as (Jx, Jy, Jz, Jx): see load_ref
    ref_array<Q>(buf, g.pop, 0)[((long long)(z * g.ny + y) * g.px + x0) >> 1] = J;
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

// Partial sums of (rho - 1, rho u) per block, fixed order.  Each block takes
// whole (y, z) rows (row = blockIdx.x + k * gridDim.x) and its threads stride
// along x, so cells are decoded with one division per row.  A cell's moments
// are FP32 sums of its 27 (15) stored deviations; the running sums across
// cells are FP64 (FP64 is slow on this GPU, so it is kept to 4 adds per cell).
template <int Q, typename T>
__global__ void __launch_bounds__(kRedThreads) conservation_kernel(const T *__restrict__ buf,
                                                                   const StepArgs a,
                                                                   double *__restrict__ part) {
    const long long N = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long rows = (long long)a.g.ny * a.g.nz;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = int(row % a.g.ny), z = int(row / a.g.ny);
        for (int x = threadIdx.x; x < a.g.nx; x += blockDim.x) {
            float f[Q];
            gather<Q, T>(buf, a.g, pull_sources(a.g, x, y, z), f);
            float drho, jx, jy, jz, Fx, Fy, Fz;
            moments<Q>(f, drho, jx, jy, jz);
            cell_force(a, row * a.g.nx + x, N, Fx, Fy, Fz);
            acc[0] += double(drho);
            acc[1] += double(jx + 0.5f * Fx);
            acc[2] += double(jy + 0.5f * Fy);
            acc[3] += double(jz + 0.5f * Fz);
        }
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

// Launchers.  The kernels_q27_*.cu and kernels_q15.cu units hold their
// explicit instantiations; api.cu sees them through the extern declarations
// below.
inline unsigned long long splat_bits(float v) {
    unsigned int u;
    memcpy(&u, &v, 4);
    return (unsigned long long)u << 32 | u;
}

// weighted: for collide27_g on weight-scaled inputs, (1 - omega) / 216.
inline PackedRates packed_rates(const StepArgs &a, bool weighted = false) {
    PackedRates p;
    for (int b = 0; b < 15; ++b) p.w15[b] = splat_bits(a.w[b] * k15_inv(b));
    for (int b = 0; b < 27; ++b) {
        const float w = a.w[b], nw = -a.w[b];
        const float omw = weighted ? (1.0f - a.w[b]) / 216.0f : 1.0f - a.w[b];
        unsigned int uw, unw, uomw;
        memcpy(&uw, &w, 4);
        memcpy(&unw, &nw, 4);
        memcpy(&uomw, &omw, 4);
        p.w[b] = (unsigned long long)uw << 32 | uw;
        p.nw[b] = (unsigned long long)unw << 32 | unw;
        p.omw[b] = (unsigned long long)uomw << 32 | uomw;
    }
    return p;
}

// D3Q27: the rates from the trace on (omega_9 .. omega_26) are all exactly
// 1, the paper's choice for every non-shear moment, so the pair kernels can
// take the kEq form of the relaxation (relax27: the same arithmetic, with
// the work that only fed those moments dropped).
inline bool higher_rates_are_one(const StepArgs &a) {
    for (int b = 9; b < 27; ++b)
        if (a.w[b] != 1.0f) return false;
    return true;
}

// The two-cells-per-thread kernels serve grids with even nx (D3Q27 and
// D3Q15); odd nx takes the one-cell kernel.
template <int Q, typename T>
cudaError_t launch_step(const void *fin, void *fout, const StepArgs &a, cudaStream_t st) {
    StepIO<T> io;
    for (int q = 0; q < 27; ++q) {
        io.in[q] = static_cast<const T *>(fin) + (q < Q ? q * a.g.pop : 0);
        io.out[q] = static_cast<T *>(fout) + (q < Q ? q * a.g.pop : 0);
    }
    io.ref_in = Storage<T>::kRef ? ref_array<Q>(static_cast<const T *>(fin), a.g.pop, 0) : nullptr;
    io.ref_out = Storage<T>::kRef ? ref_array<Q>(static_cast<T *>(fout), a.g.pop, 0) : nullptr;
    const bool walls = a.g.bc != 0;
    if constexpr (std::is_same<T, float>::value) {
        if (a.sr32) {  // stochastically rounded FP32 update: the one-cell kernel, any nx
            const CellLaunch L = cell_launch(a.g);
            if (walls)
                step_kernel<Q, T, true, true><<<L.grid, L.block, 0, st>>>(io, a);
            else
                step_kernel<Q, T, false, true><<<L.grid, L.block, 0, st>>>(io, a);
            return cudaGetLastError();
        }
    }
    if constexpr (Q == 27) {
        if (a.g.nx % 2 == 0) {
            Grid half = a.g;
            half.nx = a.g.nx / 2;
            const CellLaunch L = cell_launch(half);
            const PackedRates pr = packed_rates(a, kFoldedLoad<27, T>());
            const bool eq = higher_rates_are_one(a);
            if (walls && eq)
                step2_kernel<T, true, true><<<L.grid, L.block, 0, st>>>(io, a, pr);
            else if (walls)
                step2_kernel<T, true, false><<<L.grid, L.block, 0, st>>>(io, a, pr);
            else if (eq)
                step2_kernel<T, false, true><<<L.grid, L.block, 0, st>>>(io, a, pr);
            else
                step2_kernel<T, false, false><<<L.grid, L.block, 0, st>>>(io, a, pr);
            return cudaGetLastError();
        }
    } else {
        if (a.g.nx % 2 == 0) {
            Grid half = a.g;
            half.nx = a.g.nx / 2;
            const CellLaunch L = cell_launch(half);
            const PackedRates pr = packed_rates(a);
            if (walls && a.has_force)
                step2_q15_kernel<T, true, true><<<L.grid, L.block, 0, st>>>(io, a, pr);
            else if (walls)
                step2_q15_kernel<T, true, false><<<L.grid, L.block, 0, st>>>(io, a, pr);
            else if (a.has_force)
                step2_q15_kernel<T, false, true><<<L.grid, L.block, 0, st>>>(io, a, pr);
            else
                step2_q15_kernel<T, false, false><<<L.grid, L.block, 0, st>>>(io, a, pr);
            return cudaGetLastError();
        }
    }
    {
        const CellLaunch L = cell_launch(a.g);
        if (walls)
            step_kernel<Q, T, true><<<L.grid, L.block, 0, st>>>(io, a);
        else
            step_kernel<Q, T, false><<<L.grid, L.block, 0, st>>>(io, a);
    }
    return cudaGetLastError();
}

template <int Q, typename T, bool kEq, bool kForce>
void launch_aa_kernels(const StepIO<T> &io, const StepArgs &a, const PackedRates &pr, bool even,
                       const CellLaunch &L, cudaStream_t st) {
    if (even && a.g.bc)
        aa_even_kernel<Q, T, true, kEq, kForce><<<L.grid, L.block, 0, st>>>(io, a, pr);
    else if (even)
        aa_even_kernel<Q, T, false, kEq, kForce><<<L.grid, L.block, 0, st>>>(io, a, pr);
    else if (a.g.bc)
        aa_odd_kernel<Q, T, true, kEq, kForce><<<L.grid, L.block, 0, st>>>(io, a, pr);
    else
        aa_odd_kernel<Q, T, false, kEq, kForce><<<L.grid, L.block, 0, st>>>(io, a, pr);
}

// One in-place (AA) step on buffer buf: even (kAANatural -> kAASwapped) or
// odd (kAASwapped -> kAANatural).  nx must be even.  D3Q27 takes the rate-1
// form when omega_9..26 are all 1; D3Q15 the force-free cascade when there is
// no force.
template <int Q, typename T>
cudaError_t launch_step_aa(void *buf, const StepArgs &a, bool even, cudaStream_t st) {
    StepIO<T> io;
    for (int q = 0; q < 27; ++q) {
        io.in[q] = static_cast<const T *>(buf) + (q < Q ? q * a.g.pop : 0);
        io.out[q] = static_cast<T *>(buf) + (q < Q ? q * a.g.pop : 0);
    }
    // BF16 references: array 0 for the natural layout, 1 for the swapped one
    io.ref_in = Storage<T>::kRef ? ref_array<Q>(static_cast<const T *>(buf), a.g.pop, even ? 0 : 1)
                                 : nullptr;
    io.ref_out = Storage<T>::kRef ? ref_array<Q>(static_cast<T *>(buf), a.g.pop, even ? 1 : 0)
                                  : nullptr;
    Grid half = a.g;
    half.nx = a.g.nx / 2;
    const CellLaunch L = cell_launch(half);
    const PackedRates pr = packed_rates(a, kFoldedLoad<Q, T>());
    if constexpr (Q == 27) {
        if (higher_rates_are_one(a))
            launch_aa_kernels<Q, T, true, true>(io, a, pr, even, L, st);
        else
            launch_aa_kernels<Q, T, false, true>(io, a, pr, even, L, st);
    } else {
        if (a.has_force)
            launch_aa_kernels<Q, T, false, true>(io, a, pr, even, L, st);
        else
            launch_aa_kernels<Q, T, false, false>(io, a, pr, even, L, st);
    }
    return cudaGetLastError();
}

// BF16: the references of the state being loaded, before its values.
template <int Q, typename T>
cudaError_t launch_ref_init(T *buf, const Grid &g, const double *u, const double *f,
                            cudaStream_t st) {
    Grid half = g;
    half.nx = (g.nx + 1) / 2;
    const CellLaunch L = cell_launch(half);
    ref_init_kernel<Q, T><<<L.grid, L.block, 0, st>>>(buf, g, u, f);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_init(void *buf, const StepArgs &a, const double *rho, const double *u,
                        cudaStream_t st) {
    if constexpr (Storage<T>::kRef) {
        const cudaError_t e = launch_ref_init<Q, T>(static_cast<T *>(buf), a.g, u, nullptr, st);
        if (e != cudaSuccess) return e;
    }
    const CellLaunch L = cell_launch(a.g);
    init_kernel<Q, T><<<L.grid, L.block, 0, st>>>(static_cast<T *>(buf), a, rho, u);
    return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_set_state(void *buf, const Grid &g, const double *f, cudaStream_t st) {
    if constexpr (Storage<T>::kRef) {
        const cudaError_t e = launch_ref_init<Q, T>(static_cast<T *>(buf), g, nullptr, f, st);
        if (e != cudaSuccess) return e;
    }
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

// Number of partial-sum blocks the conservation reduction uses: one per
// (y, z) row up to kRedMaxBlocks.
inline int conservation_blocks(const Grid &g) {
    long long b = (long long)g.ny * g.nz;
    if (b > kRedMaxBlocks) b = kRedMaxBlocks;
    if (b < 1) b = 1;
    return int(b);
}

#define LBM_INSTANTIATE_1(EXT, Q, T)                                                             \
    EXT template cudaError_t launch_step<Q, T>(const void *, void *, const StepArgs &,          \
                                               cudaStream_t);                                  \
    EXT template cudaError_t launch_step_aa<Q, T>(void *, const StepArgs &, bool, cudaStream_t);  \
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
