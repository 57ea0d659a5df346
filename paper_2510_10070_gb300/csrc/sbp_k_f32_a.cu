// sbp_k_f32_a.cu — instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET(float, f32, 2)
SBP_DEFINE_SET(float, f32, 3)
SBP_DEFINE_SET(float, f32, 4)
SBP_DEFINE_SET(float, f32, 6)
SBP_DEFINE_SET(float, f32, 8)
SBP_DEFINE_SET(float, f32, 12)
}  // namespace sbp
