// Check-node pass kernels with FP16 message storage.
#include "check_pass.cuh"

namespace qc {
void *cn_kernel_f16(int maxdeg, int nt) { return cn_kernel_select<__half>(maxdeg, nt); }
void cn_smem_cap_f16(int cap) { cn_raise_smem_cap<__half>(cap); }
}  // namespace qc
