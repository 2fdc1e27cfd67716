// Explicit instantiation of the D3Q15 adjoint, its seeds and the
// kinetic-energy reduction (FP32, FP16, BF16 storage).
#include "adjoint_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_ADJOINT(, 15, float)
LBM_INSTANTIATE_ADJOINT(, 15, __half)
LBM_INSTANTIATE_ADJOINT(, 15, __nv_bfloat16)
}  // namespace lbm
