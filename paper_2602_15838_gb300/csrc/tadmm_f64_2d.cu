// Explicit instantiation of the batched ADMM path for double, (NX, NU, DP) = (4, 2, 2).
#include "tadmm_kernels.cuh"

namespace tadmm {
template struct Impl<double, 4, 2, 2>;
}  // namespace tadmm
