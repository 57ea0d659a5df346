// sbp_k_f64_n1024.cu — static-length instantiations of the pass kernels (see sbp_kernels.cuh).
#include "sbp_internal.h"

namespace sbp {
SBP_DEFINE_SET_N(double, f64, 1024)
}  // namespace sbp
