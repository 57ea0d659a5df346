// sbp_k_f32_n512.cu — static-length instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET_N(float, f32, 512)
SBP_DEFINE_ZVAR(float, f32, 512, 8, 1)
SBP_DEFINE_ZPAD(float, f32, 512, 16)
}  // namespace sbp
