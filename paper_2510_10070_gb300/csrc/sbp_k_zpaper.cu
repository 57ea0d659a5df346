// sbp_k_zpaper.cu — paper-parameter z-pass instantiations (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_ZPAPER(float, f32, 32, 16)
SBP_DEFINE_ZPAPER(float, f32, 64, 16)
SBP_DEFINE_ZPAPER(float, f32, 128, 16)
SBP_DEFINE_ZPAPER(float, f32, 256, 16)
SBP_DEFINE_ZPAPER(float, f32, 512, 16)
SBP_DEFINE_ZPAPER(double, f64, 32, 8)
SBP_DEFINE_ZPAPER(double, f64, 64, 8)
SBP_DEFINE_ZPAPER(double, f64, 128, 8)
SBP_DEFINE_ZPAPER(double, f64, 256, 8)
}  // namespace sbp
