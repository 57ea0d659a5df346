// sbp_k_sweep_d.cu — instantiations of the three-sweep kernels (see sbp_sweep.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SWEEP(256, 256, 64)
SBP_DEFINE_SWEEP(256, 256, 128)
}  // namespace sbp
