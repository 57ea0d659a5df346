// sbp_k_f32_n96.cu — static-length instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET_N(float, f32, 96)
SBP_DEFINE_ZPAD(float, f32, 96, 24)
}  // namespace sbp
