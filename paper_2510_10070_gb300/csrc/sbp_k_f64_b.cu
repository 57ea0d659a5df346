// sbp_k_f64_b.cu — instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET(double, f64, 8)
SBP_DEFINE_SET(double, f64, 12)
}  // namespace sbp
