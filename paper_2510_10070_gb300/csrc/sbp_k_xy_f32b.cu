// sbp_k_xy_f32b.cu — fused xy plane kernels (see sbp_xy.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_XY(float, f32, 192, 1)
SBP_DEFINE_XY(float, f32, 256, 1)
SBP_DEFINE_XY(float, f32, 512, 1)
}  // namespace sbp
