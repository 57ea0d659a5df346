// sbp_k_xy_f32c.cu — fused xy plane kernels (see sbp_xy.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_XY(float, f32, 192, 2)
SBP_DEFINE_XY(float, f32, 256, 2)
SBP_DEFINE_XY(float, f32, 512, 2)
}  // namespace sbp
