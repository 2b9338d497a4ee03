// mttkrp_bf16.cu -- MTTKRP kernel instantiations for __nv_bfloat16 factors.
#include "mttkrp_kernel.cuh"

namespace spt {
SPT_INSTANTIATE_MTTKRP_TABLE(__nv_bfloat16, mttkrp_kernel_bf16)
}  // namespace spt
