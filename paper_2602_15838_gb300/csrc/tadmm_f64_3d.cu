// Explicit instantiation of the batched ADMM path for double, (NX, NU, DP) = (6, 3, 3).
#include "tadmm_kernels.cuh"

namespace tadmm {
template struct Impl<double, 6, 3, 3>;
}  // namespace tadmm
