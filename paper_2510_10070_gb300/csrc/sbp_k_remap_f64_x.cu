// sbp_k_remap_f64_x.cu — physical-frame pass instantiations (see sbp_remap.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_REMAP_X(double, f64, 32)
SBP_DEFINE_REMAP_X(double, f64, 64)
SBP_DEFINE_REMAP_X(double, f64, 96)
SBP_DEFINE_REMAP_X(double, f64, 128)
SBP_DEFINE_REMAP_X(double, f64, 192)
SBP_DEFINE_REMAP_X(double, f64, 256)
SBP_DEFINE_REMAP_X(double, f64, 512)
SBP_DEFINE_REMAP_X(double, f64, 1024)
}  // namespace sbp
