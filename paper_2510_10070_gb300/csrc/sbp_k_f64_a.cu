// sbp_k_f64_a.cu — instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET(double, f64, 2)
SBP_DEFINE_SET(double, f64, 3)
SBP_DEFINE_SET(double, f64, 4)
SBP_DEFINE_SET(double, f64, 6)
}  // namespace sbp
