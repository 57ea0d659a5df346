// sbp_k_remap_f32_y.cu — physical-frame pass instantiations (see sbp_remap.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_REMAP_Y(float, f32, 32)
SBP_DEFINE_REMAP_Y(float, f32, 64)
SBP_DEFINE_REMAP_Y(float, f32, 96)
SBP_DEFINE_REMAP_Y(float, f32, 128)
SBP_DEFINE_REMAP_Y(float, f32, 192)
SBP_DEFINE_REMAP_Y(float, f32, 256)
SBP_DEFINE_REMAP_Y(float, f32, 512)
SBP_DEFINE_REMAP_Y(float, f32, 1024)
}  // namespace sbp
