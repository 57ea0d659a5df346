// sbp_k_f32_n32_64.cu — static-length instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET_N(float, f32, 32)
SBP_DEFINE_SET_N(float, f32, 64)
SBP_DEFINE_ZVAR(float, f32, 64, 8, 1)
SBP_DEFINE_ZPAD(float, f32, 32, 16)
SBP_DEFINE_ZPAD(float, f32, 64, 16)
}  // namespace sbp
