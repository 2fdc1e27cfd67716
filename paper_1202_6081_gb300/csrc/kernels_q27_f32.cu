// Explicit instantiation of the D3Q27 kernels (step, state, reductions,
// adjoint) with F32 storage.
#include "adjoint_kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_1(, 27, float)
LBM_INSTANTIATE_ADJOINT(, 27, float)
}  // namespace lbm
