// sbp_k_f64_c.cu — instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET(double, f64, 16)
}  // namespace sbp
