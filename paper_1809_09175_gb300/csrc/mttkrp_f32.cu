// mttkrp_f32.cu -- MTTKRP kernel instantiations for float factors.
#include "mttkrp_kernel.cuh"

namespace spt {
SPT_INSTANTIATE_MTTKRP_TABLE(float, mttkrp_kernel_f32)
}  // namespace spt
