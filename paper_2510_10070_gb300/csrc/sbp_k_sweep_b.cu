// sbp_k_sweep_b.cu — instantiations of the three-sweep kernels (see sbp_sweep.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SWEEP(128, 128, 64)
SBP_DEFINE_SWEEP(128, 128, 128)
}  // namespace sbp
