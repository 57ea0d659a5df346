// sbp_k_xy_f64.cu — fused xy plane kernels (see sbp_xy.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_XY(double, f64, 64, 1)
SBP_DEFINE_XY(double, f64, 128, 1)
SBP_DEFINE_XY(double, f64, 256, 1)
}  // namespace sbp
