// Check-node pass kernels with FP32 message storage.
#include "check_pass.cuh"

namespace qc {
void *cn_kernel_f32(int maxdeg, int nt) { return cn_kernel_select<float>(maxdeg, nt); }
void cn_smem_cap_f32(int cap) { cn_raise_smem_cap<float>(cap); }
}  // namespace qc
