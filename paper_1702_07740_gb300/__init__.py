"""qcldpc: GB300-native QC multi-edge LDPC reverse-reconciliation decoder.

The compute path is the CUDA library libqcldpc.so (C ABI in include/qcldpc.h);
``paper_1702_07740_gb300.qcldpc`` is its ctypes binding with the same names.
Importing this package loads nothing: the library is loaded (and built with
nvcc if stale) on the first call.
"""
from .qcldpc import (  # noqa: F401
    Code, Decoder, QcldpcError, create_code_from, qcldpc_bob_message_8d, qcldpc_code_info,
    qcldpc_create_code, qcldpc_decode, qcldpc_decode_soft, qcldpc_decode_workspace,
    qcldpc_destroy_code, qcldpc_last_error, qcldpc_llr_8d, qcldpc_params, qcldpc_params_init,
    qcldpc_syndrome, qcldpc_time_passes, qcldpc_bob_message, qcldpc_llr,
    qcldpc_decode_noalloc, Pool, qcldpc_pool_workspace, qcldpc_pool_load, qcldpc_pool_step,
    qcldpc_pools_step, qcldpc_pool_collect,
)
