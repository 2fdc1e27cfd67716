// Packed pair of FP32 values for Blackwell's f32x2 arithmetic
// (add/sub/mul/fma .rn.f32x2): one instruction updates the same quantity of
// two neighbouring cells, halving the issue slots of the collision, which
// otherwise bounds the step kernel.  Rounding is round-to-nearest-even per
// lane, as for scalar FP32.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct f2 {
    unsigned long long v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ explicit f2(unsigned long long x) : v(x) {}
    __device__ __forceinline__ f2(float lo, float hi) {
        asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
    }
    __device__ __forceinline__ explicit f2(float s) {
        asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(s));
    }
    __device__ __forceinline__ float lo() const {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return a;
    }
    __device__ __forceinline__ float hi() const {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
        return b;
    }
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }

// IEEE reciprocal per lane
__device__ __forceinline__ f2 vrcp(f2 a) { return f2(__frcp_rn(a.lo()), __frcp_rn(a.hi())); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }

template <typename V>
__device__ __forceinline__ V splat(float s);
template <>
__device__ __forceinline__ float splat<float>(float s) { return s; }
template <>
__device__ __forceinline__ f2 splat<f2>(float s) { return f2(s); }

}  // namespace lbm
