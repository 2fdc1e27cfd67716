// Explicit instantiations of the D3Q15 kernels (FP32, FP16, BF16 storage)
// and the final conservation reduction.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(, 15)

__global__ void __launch_bounds__(kRedThreads) reduce_final_kernel(const double *__restrict__ part,
                                                                   int blocks,
                                                                   double *__restrict__ out) {
    __shared__ double sh[4][kRedThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < blocks; b += kRedThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += part[4 * b + k];
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
        for (int k = 0; k < 4; ++k) out[k] = sh[k][0];
}

cudaError_t launch_reduce_final(const double *part, int blocks, double *out, cudaStream_t st) {
    reduce_final_kernel<<<1, kRedThreads, 0, st>>>(part, blocks, out);
    return cudaGetLastError();
}
}  // namespace lbm
