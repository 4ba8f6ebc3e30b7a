// Check-node pass kernels with int8 message storage.
#include "check_pass.cuh"

namespace qc {
void *cn_kernel_i8(int maxdeg, int nt) { return cn_kernel_select<int8_t>(maxdeg, nt); }
void cn_smem_cap_i8(int cap) { cn_raise_smem_cap<int8_t>(cap); }
}  // namespace qc
