// Lattice constants, state storage and the pull-streaming gather shared by
// the kernels of liblbm.so.
//
// State layout in HBM: structure of arrays, population-major,
//   buf[alpha][z][y][x_pitched],  alpha in the paper's velocity order,
// x fastest with a row pitch `px` (multiple of 32 elements) so that every
// row starts on a 128-byte boundary.  Each population plane is therefore a
// contiguous stream, and a warp of 32 consecutive x reads 128 bytes (FP32)
// or 64 bytes (16-bit) per population.
//
// The buffer holds the post-collision values of the previous step
// (f~ of Eq. cascadedcollision1).  A step pulls: the pre-collision value of
// population alpha at cell x is f~_alpha(x - e_alpha) (Eq. cascadedstreaming1
// read backwards), or, when x - e_alpha lies beyond a half-way bounce-back
// wall, the reversed population of the same cell, f~_opp(alpha)(x).
//
// Stored values are deviations from the lattice weights, f - w_alpha (FP32),
// or (f - w_alpha) / w_alpha (FP16/BF16).  Arithmetic on deviations keeps the
// O(1) rest state out of every rounding.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbm {

// Compile-time loop: calls f(std::integral_constant<int, i>) for i = 0..N-1,
// so table lookups on i fold to constants whatever the unroller decides
// (read the index as decltype(arg)::value inside f).
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

constexpr unsigned kWallY = 1u;
constexpr unsigned kWallZ = 2u;

// ---------------------------------------------------------------- velocities
// D3Q27 in the paper's order (Sec. 2): rest, the 6 axis vectors, the 12
// edge vectors (xy, xz, yz planes), the 8 corners.
__host__ __device__ constexpr int q27_e(int a, int c) {
    const signed char t[27][3] = {
        {0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
        {1, 1, 0},  {-1, 1, 0},  {1, -1, 0},  {-1, -1, 0}, {1, 0, 1},   {-1, 0, 1},  {1, 0, -1},
        {-1, 0, -1}, {0, 1, 1},  {0, -1, 1},  {0, 1, -1},  {0, -1, -1}, {1, 1, 1},   {-1, 1, 1},
        {1, -1, 1}, {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
    return t[a][c];
}

// D3Q15 in the paper's order (App. G): rest, 6 axis vectors, 8 corners.
__host__ __device__ constexpr int q15_e(int a, int c) {
    const signed char t[15][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 1},  {-1, 1, 1}, {1, -1, 1},
                                  {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1}, {1, -1, -1},
                                  {-1, -1, -1}};
    return t[a][c];
}

template <int Q>
__host__ __device__ constexpr int ex(int a) { return Q == 27 ? q27_e(a, 0) : q15_e(a, 0); }
template <int Q>
__host__ __device__ constexpr int ey(int a) { return Q == 27 ? q27_e(a, 1) : q15_e(a, 1); }
template <int Q>
__host__ __device__ constexpr int ez(int a) { return Q == 27 ? q27_e(a, 2) : q15_e(a, 2); }

// slot of the velocity (cx, cy, cz), -1 if it is not in the set
template <int Q>
__host__ __device__ constexpr int slot_of(int cx, int cy, int cz) {
    for (int a = 0; a < Q; ++a)
        if (ex<Q>(a) == cx && ey<Q>(a) == cy && ez<Q>(a) == cz) return a;
    return -1;
}

template <int Q>
__host__ __device__ constexpr int opposite(int a) { return slot_of<Q>(-ex<Q>(a), -ey<Q>(a), -ez<Q>(a)); }

// Lattice weights: the rest state (rho = 1, u = 0) of each lattice.
// D3Q27 factorises per axis into (1/6, 2/3, 1/6); D3Q15: 2/9, 1/9, 1/72.
template <int Q>
__host__ __device__ constexpr double weight(int a) {
    if (Q == 27) {
        const int n = ex<27>(a) * ex<27>(a) + ey<27>(a) * ey<27>(a) + ez<27>(a) * ez<27>(a);
        return n == 0 ? 8.0 / 27.0 : n == 1 ? 2.0 / 27.0 : n == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
    } else {
        const int n = ex<15>(a) * ex<15>(a) + ey<15>(a) * ey<15>(a) + ez<15>(a) * ez<15>(a);
        return n == 0 ? 2.0 / 9.0 : n == 1 ? 1.0 / 9.0 : 1.0 / 72.0;
    }
}

// ------------------------------------------------------------------- storage
template <typename T>
struct Storage;

template <>
struct Storage<float> {
    static constexpr bool kScaled = false;
    static constexpr bool kRef = false;
    __device__ __forceinline__ static float load(const float *p) { return __ldg(p); }
    __device__ __forceinline__ static void store(float *p, float v) { __stcs(p, v); }
};

template <>
struct Storage<__half> {
    static constexpr bool kScaled = true;
    static constexpr bool kRef = false;
    __device__ __forceinline__ static float load(const __half *p) {
        return __half2float(__ldg(p));
    }
    __device__ __forceinline__ static void store(__half *p, float v) {
        __stcs(reinterpret_cast<unsigned short *>(p), __half_as_ushort(__float2half_rn(v)));
    }
};

template <>
struct Storage<__nv_bfloat16> {
    static constexpr bool kScaled = true;
    static constexpr bool kRef = true;  // momentum references, see below
    __device__ __forceinline__ static float load(const __nv_bfloat16 *p) {
        return __bfloat162float(__ldg(p));
    }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, float v) {
        __stcs(reinterpret_cast<unsigned short *>(p),
               __bfloat16_as_ushort(__float2bfloat16_rn(v)));
    }
};

// ------------------------------------------------- stochastic 16-bit rounding
// The step stores 16-bit values with stochastic rounding: up or down with
// probability proportional to the distance, so each stored value is exact
// in expectation.  Round-to-nearest re-makes the rounding error of a slowly
// varying value with the same sign step after step, coherently over a
// smooth field, and that error accumulates (FP16 storage of the 512^3
// Taylor-Green flow drifts to 1.5e-3 relative error of u in 500 steps that
// way; a dither fixed per cell drifts the same way, so the random bits must
// change as the values do).  The conversions are sm_100-class
// cvt.rs.{f16x2,bf16x2}.f32, fed 32 random bits.  Each thread draws one seed
// per step (sr_seed below): a mixing hash of the raw bits of a few of its
// pre-collision (or, in some kernels, post-collision) values and of its
// position.  The bits of population q are
// the seed XORed with a distinct constant, one logic operation per stored
// pair of values.  So the rounding is a fixed function of the state: a step
// recomputed from the same state (checkpointing) and the in-place scheme
// round exactly as the two-buffer step does; and the bits change from step
// to step as the values move.

// Two multiply-xorshift rounds: every output bit depends on every input bit.
__device__ __forceinline__ unsigned sr_mix(unsigned x) {
    x *= 0x9E3779B1u;
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    return x;
}

// Seed from 64 bits of pre-collision values (the XOR of some of them) and the
// element offset of the thread's cell (pair).
__device__ __forceinline__ unsigned sr_seed(unsigned long long vals, int own) {
    const unsigned lo = static_cast<unsigned>(vals), hi = static_cast<unsigned>(vals >> 32);
    return sr_mix(lo ^ __funnelshift_l(hi, hi, 16) ^ static_cast<unsigned>(own));
}

// 32 random bits for population q: the FP16 conversion reads bits 0-12 for
// the low lane and 16-28 for the high lane, BF16 bits 0-15 and 16-31.
template <int q>
__device__ __forceinline__ unsigned sr_bits(unsigned seed) {
    return seed ^ (0x9E3779B9u * static_cast<unsigned>(q + 1));
}

// a + b rounded stochastically to FP32.  The exact sum lies between
// s = fl(a + b) and the neighbour n of s toward the residual r = (a + b) - s,
// which an error-free transformation (Knuth's two-sum, six operations, no
// contraction) gives exactly; n is taken with probability |r| / |n - s|,
// from the top 24 of the 32 random bits.  Used by the opt-in stochastically
// rounded FP32 update (LBM_F32_SR).
__device__ __forceinline__ float add_sr32(float a, float b, unsigned bits) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float r = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    if (r == 0.0f) return s;
    const float n = nextafterf(s, r > 0.0f ? INFINITY : -INFINITY);
    const float gap = fabsf(__fsub_rn(n, s));  // a power of two: exact
    const float u = __uint2float_rz(bits >> 8) * 0x1p-24f;
    return __fmul_rn(u, gap) < fabsf(r) ? n : s;
}

// (lo, hi) -> packed 16-bit pair (lo in the low half), stochastically rounded.
template <typename T>
struct PackSR;
template <>
struct PackSR<__half> {
    __device__ __forceinline__ static unsigned run(float lo, float hi, unsigned bits) {
        unsigned d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(bits));
        return d;
    }
};
template <>
struct PackSR<__nv_bfloat16> {
    __device__ __forceinline__ static unsigned run(float lo, float hi, unsigned bits) {
        unsigned d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(bits));
        return d;
    }
};
template <typename T, int q>
__device__ __forceinline__ unsigned pack_sr(float lo, float hi, unsigned seed) {
    return PackSR<T>::run(lo, hi, sr_bits<q>(seed));
}

// Deviation f - w (FP32) -> stored value (ref: the value's momentum
// reference, 0 unless the storage keeps one).
template <int Q, typename T>
__device__ __forceinline__ void store_dev(T *p, int a, float dev, float ref = 0.0f) {
    if (Storage<T>::kScaled)
        Storage<T>::store(p, dev * float(1.0 / weight<Q>(a)) - ref);
    else
        Storage<T>::store(p, dev);
}

// The step's store of population a of one cell: FP32 as is, 16-bit
// stochastically rounded (ref: as for store_dev).
template <int Q, typename T, int a>
__device__ __forceinline__ void store_dev_step(T *p, float dev, unsigned seed, float ref = 0.0f) {
    if constexpr (Storage<T>::kScaled) {
        const unsigned d =
            pack_sr<T, a>(fmaf(dev, float(1.0 / weight<Q>(a)), -ref), 0.0f, seed);
        __stcs(reinterpret_cast<unsigned short *>(p), static_cast<unsigned short>(d & 0xffffu));
    } else {
        Storage<T>::store(p, dev);
    }
}

// ---------------------------------------------------------------------- grid
// How a state buffer holds the pre-collision distributions f(x, t):
//   kPull:      post-collision values of the previous step at their own cells
//               (two-buffer pull scheme): f_a(x) = buf[a](x - e_a), or
//               buf[opp a](x) behind a bounce-back wall;
//   kAANatural: single-buffer (AA) scheme, a freshly loaded state or one
//               after an even number of in-place steps: f_a(x) = buf[a](x);
//   kAASwapped: AA scheme after an odd number of in-place steps (the last
//               one collided in place without streaming):
//               f_a(x) = buf[opp a](x - e_a), or buf[a](x) behind a wall.
constexpr int kPull = 0;
constexpr int kAANatural = 1;
constexpr int kAASwapped = 2;

struct Grid {
    int nx, ny, nz;   // cells
    int px;           // row pitch in elements
    unsigned bc;      // kWallY | kWallZ
    long long plane;  // px * ny
    long long pop;    // px * ny * nz: distance between populations
    int layout;       // kPull, kAANatural or kAASwapped (state reads and writes)
};

// ------------------------------------------------- BF16 momentum references
// BF16 keeps 8 significant bits, and (f - w)/w is O(3 |u|) in a moving flow:
// its rounding noise alone puts the velocity 1.4e-3 (relative L2) off.  So a
// BF16 state buffer stores, for every population a with one or two nonzero
// velocity components (the axis and edge populations, which carry ~95 % of
// the momentum's weight), the value relative to the linear part of the local
// equilibrium,
//     stored_a = (f_a - w_a) / w_a - e_a . J,
// where J = 3 u-bar is three times the mean velocity of the pair of cells
// (x even, x + 1) that produced the value (the cell whose collision wrote
// it).  The rest is O(u^2) plus the non-equilibrium part, an order of
// magnitude smaller, and so is its rounding.  The corners (|e|^2 = 3) keep
// (f - w)/w.  J of every pair sits in an FP32 array after the population
// planes of the buffer, float4 (Jx, Jy, Jz, Jx) per pair of the pitched row
// (Jx twice so that the pairs (Jx, Jy) and (Jz, Jx) are aligned 8-byte
// loads), 8 bytes per cell; the in-place scheme keeps two such arrays (index 0 for
// the natural layout, 1 for the swapped one).
//
// Who produced a value: the pre-collision f_a(x) is population a of the
// cell x - e_a after its collision, or, behind a bounce-back wall,
// population opp(a) of x itself, whatever the layout.  So a reader adds
// e_a . J(pair of x - e_a), or -e_a . J(pair of x) behind a wall.
template <int Q>
__host__ __device__ constexpr bool has_ref(int a) {
    return ex<Q>(a) * ex<Q>(a) + ey<Q>(a) * ey<Q>(a) + ez<Q>(a) * ez<Q>(a) <= 2 &&
           (ex<Q>(a) != 0 || ey<Q>(a) != 0 || ez<Q>(a) != 0);
}

// e_a . J with the components of population a known at compile time.
template <int Q, int a>
__device__ __forceinline__ float ref_dot(const float4 &J) {
    constexpr int cx = ex<Q>(a), cy = ey<Q>(a), cz = ez<Q>(a);
    float r = 0.0f;
    bool first = true;
    if constexpr (cx != 0) {
        r = cx > 0 ? J.x : -J.x;
        first = false;
    }
    if constexpr (cy != 0) {
        r = first ? (cy > 0 ? J.y : -J.y) : (cy > 0 ? r + J.y : r - J.y);
        first = false;
    }
    if constexpr (cz != 0) r = first ? (cz > 0 ? J.z : -J.z) : (cz > 0 ? r + J.z : r - J.z);
    return r;
}

// Reference array `which` of a state buffer of storage T (pop = elements per
// population plane, even).  Pair of the element at offset e: e >> 1 (rows
// start at even offsets).
template <int Q, typename T>
__host__ __device__ inline const float4 *ref_array(const T *buf, long long pop, int which) {
    return reinterpret_cast<const float4 *>(buf + (long long)Q * pop) + (long long)which * (pop / 2);
}
template <int Q, typename T>
__host__ __device__ inline float4 *ref_array(T *buf, long long pop, int which) {
    return reinterpret_cast<float4 *>(buf + (long long)Q * pop) + (long long)which * (pop / 2);
}

// Source coordinates of the pull for one cell.  Index 0, 1, 2 of each array
// is the velocity component -1, 0, +1; the source along an axis is the cell
// coordinate minus the component.  wall[...] is set where that source lies
// beyond a bounce-back wall.
struct PullSources {
    int xs[3];
    long long row[3][3];  // (zs * ny + ys) * px for (cy, cz)
    bool wall[3][3];      // bounce back for (cy, cz)
    long long own;        // (z * ny + y) * px + x
};

__device__ __forceinline__ PullSources pull_sources(const Grid &g, int x, int y, int z) {
    PullSources s;
    s.xs[0] = (x + 1 == g.nx) ? 0 : x + 1;
    s.xs[1] = x;
    s.xs[2] = (x == 0) ? g.nx - 1 : x - 1;
    int ys[3], zs[3];
    bool wy[3], wz[3];
    ys[1] = y;
    wy[1] = false;
    ys[0] = (y + 1 == g.ny) ? 0 : y + 1;
    wy[0] = (y + 1 == g.ny) && (g.bc & kWallY);
    ys[2] = (y == 0) ? g.ny - 1 : y - 1;
    wy[2] = (y == 0) && (g.bc & kWallY);
    zs[1] = z;
    wz[1] = false;
    zs[0] = (z + 1 == g.nz) ? 0 : z + 1;
    wz[0] = (z + 1 == g.nz) && (g.bc & kWallZ);
    zs[2] = (z == 0) ? g.nz - 1 : z - 1;
    wz[2] = (z == 0) && (g.bc & kWallZ);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s.row[j][k] = ((long long)zs[k] * g.ny + ys[j]) * g.px;
            s.wall[j][k] = wy[j] || wz[k];
        }
    s.own = ((long long)z * g.ny + y) * g.px + x;
    return s;
}

// Pre-collision deviations f_alpha(x) - w_alpha of one cell (slot order).
template <int Q, typename T>
__device__ __forceinline__ void gather(const T *__restrict__ fin, const Grid &g,
                                       const PullSources &s, float (&f)[Q]) {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int j = ey<Q>(a) + 1, k = ez<Q>(a) + 1, i = ex<Q>(a) + 1;
        const int o = opposite<Q>(a);
        long long idx;
        if (g.layout == kAANatural) {
            idx = (long long)a * g.pop + s.own;
        } else if (s.wall[j][k]) {
            idx = (long long)(g.layout == kPull ? o : a) * g.pop + s.own;
        } else {
            idx = (long long)(g.layout == kPull ? a : o) * g.pop + s.row[j][k] + s.xs[i];
        }
        float v = Storage<T>::load(fin + idx);
        if constexpr (Storage<T>::kRef) {
            if (has_ref<Q>(a)) {
                // producer: x - e_a, or x itself behind a wall (population opp(a))
                const float4 *R = ref_array<Q>(fin, g.pop, g.layout == kAASwapped ? 1 : 0);
                const long long prod = s.wall[j][k] ? s.own : s.row[j][k] + s.xs[i];
                const float4 J = __ldg(R + (prod >> 1));
                const float r = ex<Q>(a) * J.x + ey<Q>(a) * J.y + ez<Q>(a) * J.z;
                v += s.wall[j][k] ? -r : r;
            }
        }
        // the weight of a slot and of its opposite are equal
        f[a] = Storage<T>::kScaled ? v * float(weight<Q>(a)) : v;
    }
}

// Inverse of the pull: place the pre-collision values f_alpha(x) of one cell
// where the next step will read them (used to load a state; the AA scheme
// loads into its natural layout).
// With momentum references (BF16) the reference array 0 must already hold J
// of every pair (ref_init_kernel), and each value is stored relative to the
// reference of its producer, as a reader will add it back.
template <int Q, typename T>
__device__ __forceinline__ void scatter_state(T *__restrict__ buf, const Grid &g,
                                              const PullSources &s, const float (&f)[Q]) {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int j = ey<Q>(a) + 1, k = ez<Q>(a) + 1, i = ex<Q>(a) + 1;
        float ref = 0.0f;
        if constexpr (Storage<T>::kRef) {
            if (has_ref<Q>(a)) {
                const float4 *R = ref_array<Q>(static_cast<const T *>(buf), g.pop, 0);
                const long long prod = s.wall[j][k] ? s.own : s.row[j][k] + s.xs[i];
                const float4 J = R[prod >> 1];
                const float r = ex<Q>(a) * J.x + ey<Q>(a) * J.y + ez<Q>(a) * J.z;
                ref = s.wall[j][k] ? -r : r;
            }
        }
        if (g.layout != kPull) {
            store_dev<Q, T>(buf + (long long)a * g.pop + s.own, a, f[a], ref);
        } else if (s.wall[j][k]) {
            const int o = opposite<Q>(a);
            store_dev<Q, T>(buf + (long long)o * g.pop + s.own, o, f[a], ref);
        } else {
            store_dev<Q, T>(buf + (long long)a * g.pop + s.row[j][k] + s.xs[i], a, f[a], ref);
        }
    }
}

}  // namespace lbm
