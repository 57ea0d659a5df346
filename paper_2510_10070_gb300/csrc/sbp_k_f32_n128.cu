// sbp_k_f32_n128.cu — static-length instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET_N(float, f32, 128)
SBP_DEFINE_ZVAR(float, f32, 128, 8, 1)
SBP_DEFINE_ZVAR(float, f32, 128, 8, 0)
SBP_DEFINE_ZPAD(float, f32, 128, 16)
}  // namespace sbp
