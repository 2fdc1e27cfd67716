// Explicit instantiation of the D3Q27 kernels (step, state, reductions,
// adjoint) with BF16 storage.
#include "adjoint_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_1(, 27, __nv_bfloat16)
LBM_INSTANTIATE_ADJOINT(, 27, __nv_bfloat16)
}  // namespace lbm
