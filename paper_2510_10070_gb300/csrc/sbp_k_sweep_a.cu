// sbp_k_sweep_a.cu — instantiations of the three-sweep kernels (see sbp_sweep.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SWEEP(32, 32, 32)
SBP_DEFINE_SWEEP(64, 64, 32)
SBP_DEFINE_SWEEP(64, 64, 64)
}  // namespace sbp
