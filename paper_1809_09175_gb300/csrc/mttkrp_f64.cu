// mttkrp_f64.cu -- MTTKRP kernel instantiations for double factors (fp64
// accumulation and output, the precision the paper measures in, Sec. 7).
#include "mttkrp_kernel.cuh"

namespace spt {
SPT_INSTANTIATE_MTTKRP_TABLE(double, mttkrp_kernel_f64)
}  // namespace spt
