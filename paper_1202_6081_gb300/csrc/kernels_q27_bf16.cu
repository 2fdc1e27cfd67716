// Explicit instantiation of the D3Q27 kernels with BF16 storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_1(, 27, __nv_bfloat16)
}  // namespace lbm
