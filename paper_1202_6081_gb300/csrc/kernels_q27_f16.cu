// Explicit instantiation of the D3Q27 kernels (step, state, reductions,
// adjoint) with F16 storage.
#include "adjoint_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_1(, 27, __half)
LBM_INSTANTIATE_ADJOINT(, 27, __half)
}  // namespace lbm
