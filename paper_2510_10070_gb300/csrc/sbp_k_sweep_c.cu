// sbp_k_sweep_c.cu — instantiations of the three-sweep kernels (see sbp_sweep.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SWEEP(192, 192, 96)
}  // namespace sbp
