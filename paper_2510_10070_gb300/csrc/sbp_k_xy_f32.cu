// sbp_k_xy_f32.cu — fused xy plane kernels (see sbp_xy.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_XY(float, f32, 64, 1)
SBP_DEFINE_XY(float, f32, 96, 1)
SBP_DEFINE_XY(float, f32, 128, 1)
SBP_DEFINE_XY(float, f32, 128, 2)
}  // namespace sbp
