"""Thin ctypes binding of libqcldpc (include/qcldpc.h). Argument marshalling only.

Every function keeps the C name. Device buffers are torch CUDA tensors (any
dtype of the right width, contiguous); the stream defaults to torch's current
stream. All arithmetic runs in the CUDA library: if it is missing or no GPU is
visible, the compute calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

QCLDPC_OK = 0
STATUS = {
    -1: "QCLDPC_E_INVAL", -2: "QCLDPC_E_SHIFT_RANGE", -3: "QCLDPC_E_DUP_SHIFT",
    -4: "QCLDPC_E_ALIGN", -5: "QCLDPC_E_NOMEM", -6: "QCLDPC_E_CUDA",
    -7: "QCLDPC_E_TIMEOUT", -8: "QCLDPC_E_UNSUPPORTED",
}

# Every symbol include/qcldpc.h declares.
EXPORTED = [
    "qcldpc_create_code", "qcldpc_destroy_code", "qcldpc_code_info",
    "qcldpc_syndrome", "qcldpc_bob_message_8d", "qcldpc_llr_8d",
    "qcldpc_bob_message", "qcldpc_llr",
    "qcldpc_params_init", "qcldpc_decode_workspace", "qcldpc_decode",
    "qcldpc_decode_soft", "qcldpc_decode_multi_workspace", "qcldpc_decode_multi",
    "qcldpc_time_passes", "qcldpc_decode_noalloc", "qcldpc_autotune",
    "qcldpc_autotune_shapes",
    "qcldpc_pool_workspace", "qcldpc_pool_create", "qcldpc_pool_destroy", "qcldpc_pool_state",
    "qcldpc_pool_load", "qcldpc_pool_step", "qcldpc_pools_step", "qcldpc_pool_collect",
    "qcldpc_last_error",
]


class QcldpcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


class qcldpc_params(ctypes.Structure):
    _fields_ = [
        ("clip", ctypes.c_float),
        ("phi_floor", ctypes.c_float),
        ("et_start", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("msg_format", ctypes.c_int32),
        ("soft_output", ctypes.c_int32),
        ("launch_mode", ctypes.c_int32),
        ("msg_step", ctypes.c_float),
        ("layers", ctypes.c_int32),
        ("cn_threads", ctypes.c_int32),
        ("vn_nodes", ctypes.c_int32),
        ("vn_split", ctypes.c_int32),
        ("vn_pass", ctypes.c_int32),
        ("frame_groups", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqcldpc.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("QCLDPC_LIB") or _build.LIB
        if path == _build.LIB and build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libqcldpc.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        lib.qcldpc_create_code.argtypes = [i32, i32, i32, i32, vp, vp, vp, ctypes.POINTER(vp)]
        lib.qcldpc_create_code.restype = i32
        lib.qcldpc_destroy_code.argtypes = [vp]
        lib.qcldpc_destroy_code.restype = None
        lib.qcldpc_code_info.argtypes = [vp, vp, vp, vp, vp]
        lib.qcldpc_code_info.restype = i32
        lib.qcldpc_syndrome.argtypes = [vp, vp, vp, i32, vp]
        lib.qcldpc_syndrome.restype = i32
        lib.qcldpc_bob_message_8d.argtypes = [vp, vp, i64, vp, vp]
        lib.qcldpc_bob_message_8d.restype = i32
        lib.qcldpc_llr_8d.argtypes = [vp, vp, i64, ctypes.c_float, vp, vp]
        lib.qcldpc_llr_8d.restype = i32
        lib.qcldpc_bob_message.argtypes = [i32, vp, vp, i64, vp, vp]
        lib.qcldpc_bob_message.restype = i32
        lib.qcldpc_llr.argtypes = [i32, vp, vp, i64, ctypes.c_float, vp, vp]
        lib.qcldpc_llr.restype = i32
        lib.qcldpc_params_init.argtypes = [ctypes.POINTER(qcldpc_params)]
        lib.qcldpc_params_init.restype = None
        lib.qcldpc_decode_workspace.argtypes = [vp, i32, ctypes.POINTER(qcldpc_params)]
        lib.qcldpc_decode_workspace.restype = sz
        lib.qcldpc_decode.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(qcldpc_params),
                                      vp, vp, vp, vp, sz, vp]
        lib.qcldpc_decode.restype = i32
        lib.qcldpc_decode_multi_workspace.argtypes = [i32, vp, vp, ctypes.POINTER(qcldpc_params)]
        lib.qcldpc_decode_multi_workspace.restype = sz
        lib.qcldpc_decode_multi.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(qcldpc_params),
                                            vp, vp, vp, vp, sz, vp]
        lib.qcldpc_decode_multi.restype = i32
        lib.qcldpc_decode_soft.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(qcldpc_params),
                                           vp, vp, vp, vp, vp, sz, vp]
        lib.qcldpc_decode_soft.restype = i32
        lib.qcldpc_time_passes.argtypes = [vp, i32, vp, sz, i32, ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_float), vp]
        lib.qcldpc_time_passes.restype = i32
        lib.qcldpc_decode_noalloc.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(qcldpc_params),
                                              vp, vp, vp, vp]
        lib.qcldpc_decode_noalloc.restype = i32
        lib.qcldpc_autotune.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(qcldpc_params),
                                        vp, vp, vp, vp, sz, i32, ctypes.POINTER(qcldpc_params),
                                        ctypes.POINTER(ctypes.c_float), vp]
        lib.qcldpc_autotune.restype = i32
        lib.qcldpc_autotune_shapes.argtypes = [vp, i32, vp, sz, i32, ctypes.POINTER(qcldpc_params),
                                               ctypes.POINTER(qcldpc_params),
                                               ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_float), vp]
        lib.qcldpc_autotune_shapes.restype = i32
        lib.qcldpc_pool_workspace.argtypes = [vp, i32, ctypes.POINTER(qcldpc_params)]
        lib.qcldpc_pool_workspace.restype = sz
        lib.qcldpc_pool_create.argtypes = [vp, i32, i32, ctypes.POINTER(qcldpc_params), vp, sz, vp,
                                           ctypes.POINTER(vp)]
        lib.qcldpc_pool_create.restype = i32
        lib.qcldpc_pool_destroy.argtypes = [vp]
        lib.qcldpc_pool_destroy.restype = None
        lib.qcldpc_pool_state.argtypes = [vp, ctypes.POINTER(vp)]
        lib.qcldpc_pool_state.restype = i32
        lib.qcldpc_pool_load.argtypes = [vp, i32, vp, vp, vp, vp]
        lib.qcldpc_pool_load.restype = i32
        lib.qcldpc_pool_step.argtypes = [vp, i32, vp]
        lib.qcldpc_pool_step.restype = i32
        lib.qcldpc_pools_step.argtypes = [i32, vp, i32, vp]
        lib.qcldpc_pools_step.restype = i32
        lib.qcldpc_pool_collect.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        lib.qcldpc_pool_collect.restype = i32
        lib.qcldpc_last_error.argtypes = []
        lib.qcldpc_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def qcldpc_last_error() -> str:
    return load().qcldpc_last_error().decode()


def _check(status: int, where: str):
    if status != QCLDPC_OK:
        raise QcldpcError(status, where, qcldpc_last_error())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, nbytes_elem=None, name="buffer"):
    """Device pointer of a contiguous CUDA tensor (argument check only)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if nbytes_elem is not None and t.element_size() != nbytes_elem:
        raise TypeError(f"{name} must have {nbytes_elem}-byte elements")
    return ctypes.c_void_p(t.data_ptr())


def qcldpc_params_init(**overrides) -> qcldpc_params:
    p = qcldpc_params()
    load().qcldpc_params_init(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Code:
    """Owning wrapper of a qcldpc_code handle."""

    def __init__(self, handle, mb, nb, Z):
        self._h = handle
        self.mb, self.nb, self.Z = mb, nb, Z
        self.n, self.m, self.k, self.n_edges = qcldpc_code_info(self)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and _lib is not None:
            _lib.qcldpc_destroy_code(h)


def qcldpc_create_code(mb, nb, Z, circ_row, circ_col, circ_shift) -> Code:
    row = np.ascontiguousarray(circ_row, dtype=np.int32)
    col = np.ascontiguousarray(circ_col, dtype=np.int32)
    shift = np.ascontiguousarray(circ_shift, dtype=np.int32)
    if not (row.shape == col.shape == shift.shape) or row.ndim != 1:
        raise ValueError("circulant arrays must be 1-D and of equal length")
    out = ctypes.c_void_p()
    st = load().qcldpc_create_code(int(mb), int(nb), int(Z), int(row.shape[0]),
                                   row.ctypes.data_as(ctypes.c_void_p),
                                   col.ctypes.data_as(ctypes.c_void_p),
                                   shift.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out))
    _check(st, "qcldpc_create_code")
    return Code(out, int(mb), int(nb), int(Z))


def create_code_from(d: dict) -> Code:
    return qcldpc_create_code(d["mb"], d["nb"], d["Z"], d["row"], d["col"], d["shift"])


def qcldpc_destroy_code(code: Code):
    h, code._h = code._h, None
    if h is not None:
        load().qcldpc_destroy_code(h)


def qcldpc_code_info(code: Code):
    vals = [ctypes.c_int64() for _ in range(4)]
    st = load().qcldpc_code_info(code.handle, *[ctypes.byref(v) for v in vals])
    _check(st, "qcldpc_code_info")
    return tuple(v.value for v in vals)


def qcldpc_syndrome(code: Code, bits_dev, syn_dev, n_frames: int, stream=None):
    st = load().qcldpc_syndrome(code.handle, _dev(bits_dev, 4, "bits_dev"),
                                _dev(syn_dev, 4, "syn_dev"), int(n_frames), _stream(stream))
    _check(st, "qcldpc_syndrome")


def qcldpc_bob_message_8d(y_dev, bits_dev, n: int, m_dev, stream=None):
    st = load().qcldpc_bob_message_8d(_dev(y_dev, 4, "y_dev"), _dev(bits_dev, 4, "bits_dev"),
                                      int(n), _dev(m_dev, 4, "m_dev"), _stream(stream))
    _check(st, "qcldpc_bob_message_8d")


def qcldpc_llr_8d(x_dev, m_dev, n: int, snr: float, llr_dev, stream=None):
    st = load().qcldpc_llr_8d(_dev(x_dev, 4, "x_dev"), _dev(m_dev, 4, "m_dev"), int(n),
                              float(snr), _dev(llr_dev, 4, "llr_dev"), _stream(stream))
    _check(st, "qcldpc_llr_8d")


def qcldpc_bob_message(d: int, y_dev, bits_dev, n: int, m_dev, stream=None):
    st = load().qcldpc_bob_message(int(d), _dev(y_dev, 4, "y_dev"), _dev(bits_dev, 4, "bits_dev"),
                                   int(n), _dev(m_dev, 4, "m_dev"), _stream(stream))
    _check(st, "qcldpc_bob_message")


def qcldpc_llr(d: int, x_dev, m_dev, n: int, snr: float, llr_dev, stream=None):
    st = load().qcldpc_llr(int(d), _dev(x_dev, 4, "x_dev"), _dev(m_dev, 4, "m_dev"), int(n),
                           float(snr), _dev(llr_dev, 4, "llr_dev"), _stream(stream))
    _check(st, "qcldpc_llr")


def qcldpc_decode_workspace(code: Code, n_frames: int, params: qcldpc_params | None = None) -> int:
    p = ctypes.byref(params) if params is not None else None
    return int(load().qcldpc_decode_workspace(code.handle, int(n_frames), p))


def qcldpc_decode(code: Code, llr_dev, syn_dev, n_frames: int, max_iter: int,
                  params: qcldpc_params | None, key_bits_dev, converged_dev, iters_dev,
                  workspace_dev, workspace_bytes: int, stream=None):
    p = ctypes.byref(params) if params is not None else None
    st = load().qcldpc_decode(code.handle, _dev(llr_dev, 4, "llr_dev"),
                              _dev(syn_dev, 4, "syn_dev"), int(n_frames), int(max_iter), p,
                              _dev(key_bits_dev, 4, "key_bits_dev"),
                              _dev(converged_dev, 4, "converged_dev"),
                              _dev(iters_dev, 4, "iters_dev"), _dev(workspace_dev, None, "workspace"),
                              int(workspace_bytes), _stream(stream))
    _check(st, "qcldpc_decode")


def qcldpc_decode_soft(code: Code, llr_dev, syn_dev, n_frames: int, max_iter: int,
                       params: qcldpc_params, key_bits_dev, converged_dev, iters_dev,
                       posterior_dev, workspace_dev, workspace_bytes: int, stream=None):
    st = load().qcldpc_decode_soft(code.handle, _dev(llr_dev, 4, "llr_dev"),
                                   _dev(syn_dev, 4, "syn_dev"), int(n_frames), int(max_iter),
                                   ctypes.byref(params), _dev(key_bits_dev, 4, "key_bits_dev"),
                                   _dev(converged_dev, 4, "converged_dev"),
                                   _dev(iters_dev, 4, "iters_dev"),
                                   _dev(posterior_dev, 4, "posterior_dev"),
                                   _dev(workspace_dev, None, "workspace"), int(workspace_bytes),
                                   _stream(stream))
    _check(st, "qcldpc_decode_soft")


def _ptr_array(items, what):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = _dev(t, None, what).value if t is not None else None
    return arr


def qcldpc_decode_multi_workspace(codes: list, n_frames: list, params: qcldpc_params | None = None) -> int:
    hs = (ctypes.c_void_p * len(codes))(*[c.handle for c in codes])
    nf = (ctypes.c_int * len(codes))(*[int(f) for f in n_frames])
    p = ctypes.byref(params) if params is not None else None
    return int(load().qcldpc_decode_multi_workspace(len(codes), hs, nf, p))


def qcldpc_decode_multi(codes: list, llr_devs: list, syn_devs: list, n_frames: list, max_iter: int,
                        params: qcldpc_params | None, key_bits_devs: list, converged_devs: list,
                        iters_devs: list, workspace_dev, workspace_bytes: int, stream=None):
    n = len(codes)
    hs = (ctypes.c_void_p * n)(*[c.handle for c in codes])
    nf = (ctypes.c_int * n)(*[int(f) for f in n_frames])
    p = ctypes.byref(params) if params is not None else None
    st = load().qcldpc_decode_multi(n, hs, _ptr_array(llr_devs, "llr_dev"), _ptr_array(syn_devs, "syn_dev"),
                                    nf, int(max_iter), p, _ptr_array(key_bits_devs, "key_bits_dev"),
                                    _ptr_array(converged_devs, "converged_dev"),
                                    _ptr_array(iters_devs, "iters_dev"), _dev(workspace_dev, None, "workspace"),
                                    int(workspace_bytes), _stream(stream))
    _check(st, "qcldpc_decode_multi")


def qcldpc_time_passes(code: Code, n_frames: int, workspace_dev, workspace_bytes: int,
                       reps: int, stream=None):
    """Mean (check-node ms, variable-node ms) of replayed decoder passes."""
    cn, vn = ctypes.c_float(), ctypes.c_float()
    st = load().qcldpc_time_passes(code.handle, int(n_frames), _dev(workspace_dev, None, "workspace"),
                                   int(workspace_bytes), int(reps), ctypes.byref(cn),
                                   ctypes.byref(vn), _stream(stream))
    _check(st, "qcldpc_time_passes")
    return cn.value, vn.value


AUTOTUNE_CANDIDATES = ("flooding", "layered 2 groups", "layered 7 groups",
                       "layered min(mb,64) groups")


def qcldpc_autotune(code: Code, llr_dev, syn_dev, n_frames: int, max_iter: int,
                    params: qcldpc_params | None, key_bits_dev, converged_dev, iters_dev,
                    workspace_dev, workspace_bytes: int, reps: int = 3, stream=None):
    """Fastest schedule for the sample batch: (best params, {candidate: ms})."""
    best = qcldpc_params()
    times = (ctypes.c_float * 4)()
    p = ctypes.byref(params) if params is not None else None
    st = load().qcldpc_autotune(code.handle, _dev(llr_dev, 4, "llr_dev"), _dev(syn_dev, 4, "syn_dev"),
                                int(n_frames), int(max_iter), p, _dev(key_bits_dev, 4, "key_bits_dev"),
                                _dev(converged_dev, 4, "converged_dev"), _dev(iters_dev, 4, "iters_dev"),
                                _dev(workspace_dev, None, "workspace"), int(workspace_bytes), int(reps),
                                ctypes.byref(best), times, _stream(stream))
    _check(st, "qcldpc_autotune")
    return best, {name: times[i] for i, name in enumerate(AUTOTUNE_CANDIDATES)
                  if times[i] == times[i]}


# Launch-shape candidates of qcldpc_autotune_shapes, in its timing order.
SHAPE_CN_THREADS = tuple(32 * (i + 1) for i in range(8))
SHAPE_VN = ((1, 1), (2, 1), (3, 1), (1, 2), (2, 2), (3, 2))  # (vn_nodes, vn_split)


def qcldpc_autotune_shapes(code: Code, n_frames: int, workspace_dev, workspace_bytes: int,
                           params: qcldpc_params | None = None, reps: int = 5, stream=None):
    """Fastest launch shapes on the state of the last flooding decode:
    (best params, {cn_threads: ms}, {(vn_nodes, vn_split): ms})."""
    best = qcldpc_params()
    tc = (ctypes.c_float * len(SHAPE_CN_THREADS))()
    tv = (ctypes.c_float * len(SHAPE_VN))()
    p = ctypes.byref(params) if params is not None else None
    st = load().qcldpc_autotune_shapes(code.handle, int(n_frames), _dev(workspace_dev, None, "workspace"),
                                       int(workspace_bytes), int(reps), p, ctypes.byref(best), tc, tv,
                                       _stream(stream))
    _check(st, "qcldpc_autotune_shapes")
    return (best, {c: tc[i] for i, c in enumerate(SHAPE_CN_THREADS)},
            {c: tv[i] for i, c in enumerate(SHAPE_VN)})


def qcldpc_decode_noalloc(code: Code, llr_dev, syn_dev, n_frames: int, max_iter: int,
                          params: qcldpc_params | None, key_bits_dev, converged_dev, iters_dev,
                          stream=None):
    """qcldpc_decode with the library's static scratch instead of a workspace."""
    p = ctypes.byref(params) if params is not None else None
    st = load().qcldpc_decode_noalloc(code.handle, _dev(llr_dev, 4, "llr_dev"),
                                      _dev(syn_dev, 4, "syn_dev"), int(n_frames), int(max_iter), p,
                                      _dev(key_bits_dev, 4, "key_bits_dev"),
                                      _dev(converged_dev, 4, "converged_dev"),
                                      _dev(iters_dev, 4, "iters_dev"), _stream(stream))
    _check(st, "qcldpc_decode_noalloc")


class MultiDecoder:
    """Owner of the device buffers of a batched decode of several codes
    (``qcldpc_decode_multi``): ``codes[c]`` decodes ``n_frames[c]`` frames;
    ``keys[c]``, ``converged[c]`` and ``iters[c]`` hold its outputs."""

    def __init__(self, codes: list, n_frames: list, params: qcldpc_params | None = None, device=None):
        import torch
        self.codes, self.n_frames = list(codes), [int(f) for f in n_frames]
        self.params = params if params is not None else qcldpc_params_init()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.ws_bytes = qcldpc_decode_multi_workspace(self.codes, self.n_frames, self.params)
        if self.ws_bytes == 0:
            raise QcldpcError(-1, "qcldpc_decode_multi_workspace", "invalid arguments")
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.keys = [torch.zeros(max(f, 1) * ((c.k + 31) // 32), dtype=torch.int32, device=dev)
                     for c, f in zip(self.codes, self.n_frames)]
        self.converged = [torch.zeros(max(f, 1), dtype=torch.int32, device=dev) for f in self.n_frames]
        self.iters = [torch.zeros(max(f, 1), dtype=torch.int32, device=dev) for f in self.n_frames]

    def decode(self, llr_devs: list, syn_devs: list, max_iter: int, stream=None):
        qcldpc_decode_multi(self.codes, llr_devs, syn_devs, self.n_frames, max_iter, self.params, self.keys,
                            self.converged, self.iters, self.workspace, self.ws_bytes, stream)


class Decoder:
    """Convenience owner of the device buffers one decode batch needs.

    Holds the code, a workspace and the output tensors for ``n_frames``
    frames; ``decode`` enqueues ``qcldpc_decode`` (or the soft variant).
    """

    def __init__(self, code: Code, n_frames: int, params: qcldpc_params | None = None,
                 soft: bool = False, device=None):
        import torch
        self.code = code
        self.n_frames = int(n_frames)
        self.params = params if params is not None else qcldpc_params_init()
        if soft:
            self.params.soft_output = 1
        self.soft = soft
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.ws_bytes = qcldpc_decode_workspace(code, self.n_frames, self.params)
        self.workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        wk = (code.k + 31) // 32
        self.keys = torch.zeros(self.n_frames * wk, dtype=torch.int32, device=dev)
        self.converged = torch.zeros(self.n_frames, dtype=torch.int32, device=dev)
        self.iters = torch.zeros(self.n_frames, dtype=torch.int32, device=dev)
        self.posterior = (torch.zeros(self.n_frames * code.n, dtype=torch.float32, device=dev)
                          if soft else None)

    def decode(self, llr_dev, syn_dev, max_iter: int, stream=None):
        if self.soft:
            qcldpc_decode_soft(self.code, llr_dev, syn_dev, self.n_frames, max_iter,
                               self.params, self.keys, self.converged, self.iters,
                               self.posterior, self.workspace, self.ws_bytes, stream)
        else:
            qcldpc_decode(self.code, llr_dev, syn_dev, self.n_frames, max_iter, self.params,
                          self.keys, self.converged, self.iters, self.workspace,
                          self.ws_bytes, stream)


# ---------------------------------------------------------------- pools

def qcldpc_pool_workspace(code: Code, n_slots: int, params: qcldpc_params | None = None) -> int:
    p = ctypes.byref(params) if params is not None else None
    return int(load().qcldpc_pool_workspace(code.handle, int(n_slots), p))


class Pool:
    """Owning wrapper of a qcldpc_pool: n_slots frame slots of one code.

    Holds its workspace tensor; ``state`` is a view of the device slot states
    (0 free, 1 running, 2 stopped).
    """

    def __init__(self, code: Code, n_slots: int, max_iter: int,
                 params: qcldpc_params | None = None, stream=None, device=None):
        import torch
        self.code, self.n_slots, self.max_iter = code, int(n_slots), int(max_iter)
        self.params = params if params is not None else qcldpc_params_init()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.ws_bytes = qcldpc_pool_workspace(code, self.n_slots, self.params)
        if self.ws_bytes == 0:
            raise QcldpcError(-1, "qcldpc_pool_workspace", "invalid arguments")
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        st = load().qcldpc_pool_create(code.handle, self.n_slots, self.max_iter,
                                       ctypes.byref(self.params), _dev(self.workspace, None, "ws"),
                                       self.ws_bytes, _stream(stream), ctypes.byref(h))
        _check(st, "qcldpc_pool_create")
        self._h = h
        ptr = ctypes.c_void_p()
        _check(load().qcldpc_pool_state(self._h, ctypes.byref(ptr)), "qcldpc_pool_state")
        off = ptr.value - self.workspace.data_ptr()
        self.state = self.workspace[off: off + 4 * self.n_slots].view(torch.int32)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and _lib is not None:
            _lib.qcldpc_pool_destroy(h)


def qcldpc_pool_load(pool: Pool, n: int, slots_dev, llr_dev, syn_dev, stream=None):
    st = load().qcldpc_pool_load(pool.handle, int(n), _dev(slots_dev, 4, "slots_dev"),
                                 _dev(llr_dev, 4, "llr_dev"), _dev(syn_dev, 4, "syn_dev"),
                                 _stream(stream))
    _check(st, "qcldpc_pool_load")


def qcldpc_pool_step(pool: Pool, n_passes: int, stream=None):
    _check(load().qcldpc_pool_step(pool.handle, int(n_passes), _stream(stream)), "qcldpc_pool_step")


def qcldpc_pools_step(pools, n_passes: int, stream=None):
    arr = (ctypes.c_void_p * len(pools))(*[p.handle.value for p in pools])
    st = load().qcldpc_pools_step(len(pools), ctypes.cast(arr, ctypes.c_void_p), int(n_passes),
                                  _stream(stream))
    _check(st, "qcldpc_pools_step")


def qcldpc_pool_collect(pool: Pool, n: int, slots_dev, key_bits_dev, converged_dev, iters_dev,
                        stream=None):
    st = load().qcldpc_pool_collect(pool.handle, int(n), _dev(slots_dev, 4, "slots_dev"),
                                    _dev(key_bits_dev, 4, "key_bits_dev"),
                                    _dev(converged_dev, 4, "converged_dev"),
                                    _dev(iters_dev, 4, "iters_dev"), _stream(stream))
    _check(st, "qcldpc_pool_collect")
