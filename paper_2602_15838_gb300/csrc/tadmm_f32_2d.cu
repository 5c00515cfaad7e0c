// Explicit instantiation of the batched ADMM path for float, (NX, NU, DP) = (4, 2, 2).
#include "tadmm_kernels.cuh"

namespace tadmm {
template struct Impl<float, 4, 2, 2>;
}  // namespace tadmm
