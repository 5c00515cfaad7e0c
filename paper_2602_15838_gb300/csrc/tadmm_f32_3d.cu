// Explicit instantiation of the batched ADMM path for float, (NX, NU, DP) = (6, 3, 3).
#include "tadmm_kernels.cuh"

namespace tadmm {
template struct Impl<float, 6, 3, 3>;
}  // namespace tadmm
