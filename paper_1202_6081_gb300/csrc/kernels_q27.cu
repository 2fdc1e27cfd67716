// Explicit instantiations of the D3Q27 kernels (FP32, FP16, BF16 storage).
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE(, 27)
}  // namespace lbm
