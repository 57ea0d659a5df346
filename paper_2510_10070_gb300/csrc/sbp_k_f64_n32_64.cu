// sbp_k_f64_n32_64.cu — static-length instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET_N(double, f64, 32)
SBP_DEFINE_SET_N(double, f64, 64)
SBP_DEFINE_ZPAD(double, f64, 32, 8)
SBP_DEFINE_ZPAD(double, f64, 64, 8)
}  // namespace sbp
