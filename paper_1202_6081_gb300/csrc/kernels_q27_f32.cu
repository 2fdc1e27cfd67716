// Explicit instantiation of the D3Q27 kernels with F32 storage.
#include "kernels.cuh"

namespace lbm {
LBM_INSTANTIATE_1(, 27, float)
}  // namespace lbm
