// sbp_k_f32_c.cu — instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET(float, f32, 24)
}  // namespace sbp
