// Explicit instantiation of the batched ADMM path in double-float arithmetic, (NX, NU, DP) = (4, 2, 2).
#include "tadmm_kernels.cuh"

namespace tadmm {
template struct Impl<df64, 4, 2, 2>;
}  // namespace tadmm
