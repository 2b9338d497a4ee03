// mttkrp_f16.cu -- MTTKRP kernel instantiations for __half factors.
#include "mttkrp_kernel.cuh"

namespace spt {
SPT_INSTANTIATE_MTTKRP_TABLE(__half, mttkrp_kernel_f16)
}  // namespace spt
