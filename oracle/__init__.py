"""Plain FP64 CPU oracle for QC multi-edge LDPC reverse reconciliation.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA decoder never
imports this package and this package imports nothing from it.

The arithmetic lives in ``qcldpc_oracle.c`` (plain C99, IEEE double, no
fused multiply-add); this module only compiles it with gcc and marshals numpy
arrays. Brute-force references for tiny codes are in ``oracle.brute``.

Paper: arXiv 1702.07740. Sec. III-C (QC expansion), Sec. II-C (Bob's message
and the d-dimensional division), Algorithm 1 (sum-product decoding).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcldpc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

# Default numerical guards of the decoder (clip level and Phi floor).
CLIP = 15.0
XMIN = 1e-6


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32, i64, dbl, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.orc_expand.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp]
        lib.orc_expand.restype = i32
        lib.orc_syndrome.argtypes = [i64, i64, vp, vp, vp, vp]
        lib.orc_syndrome.restype = None
        lib.orc_cd_mul.argtypes = [vp, vp, vp, i32]
        lib.orc_cd_mul.restype = None
        lib.orc_bob_message.argtypes = [i32, i64, vp, vp, vp]
        lib.orc_bob_message.restype = i32
        lib.orc_llr.argtypes = [i32, i64, vp, vp, dbl, vp]
        lib.orc_llr.restype = i32
        lib.orc_phi.argtypes = [dbl]
        lib.orc_phi.restype = dbl
        lib.orc_decode.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, i32,
                                   dbl, dbl, vp, vp, vp, vp]
        lib.orc_decode.restype = i32
        lib.orc_decode_layered.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp, i32,
                                           i32, dbl, dbl, vp, vp, vp, vp]
        lib.orc_decode_layered.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Code:
    """Expanded QC code: the edge list of H (Sec. III-C).

    ``row, col, shift`` list the circulants of the base matrix; circulant h
    yields edges e = h*Z + i between check row*Z + i and variable
    col*Z + (i + shift) mod Z.
    """

    def __init__(self, mb, nb, Z, row, col, shift):
        self.mb, self.nb, self.Z = int(mb), int(nb), int(Z)
        self.row = np.ascontiguousarray(row, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.shift = np.ascontiguousarray(shift, dtype=np.int32)
        self.n = self.nb * self.Z
        self.m = self.mb * self.Z
        self.k = self.n - self.m
        nc = len(self.row)
        self.n_edges = nc * self.Z
        self.edge_cn = np.zeros(max(self.n_edges, 1), dtype=np.int64)
        self.edge_vn = np.zeros(max(self.n_edges, 1), dtype=np.int64)
        rc = _load().orc_expand(self.mb, self.nb, self.Z, nc, _ptr(self.row),
                                _ptr(self.col), _ptr(self.shift),
                                _ptr(self.edge_cn), _ptr(self.edge_vn))
        if rc != 0:
            raise ValueError("circulant entry out of range")
        self.edge_cn = self.edge_cn[: self.n_edges]
        self.edge_vn = self.edge_vn[: self.n_edges]

    @classmethod
    def from_dict(cls, d):
        return cls(d["mb"], d["nb"], d["Z"], d["row"], d["col"], d["shift"])

    def dense(self) -> np.ndarray:
        """Dense H over GF(2) (small codes only)."""
        H = np.zeros((self.m, self.n), dtype=np.uint8)
        for c, v in zip(self.edge_cn, self.edge_vn):
            H[c, v] ^= 1
        return H


def syndrome(code: Code, bits: np.ndarray) -> np.ndarray:
    """s = H x (mod 2) for one frame of 0/1 bytes."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    assert bits.shape == (code.n,)
    syn = np.zeros(code.m, dtype=np.uint8)
    _load().orc_syndrome(code.m, code.n_edges, _ptr(code.edge_cn),
                         _ptr(code.edge_vn), _ptr(bits), _ptr(syn))
    return syn


def cd_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Cayley-Dickson product of two d-vectors, d in {1,2,4,8}."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    d = a.shape[0]
    assert d in (1, 2, 4, 8) and b.shape == (d,)
    out = np.zeros(d, dtype=np.float64)
    _load().orc_cd_mul(_ptr(a), _ptr(b), _ptr(out), d)
    return out


def bob_message(y: np.ndarray, bits: np.ndarray, d: int = 8) -> np.ndarray:
    """Bob's public message M = U Y per block of d (U_j = (-1)^{C_j})."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    m = np.zeros_like(y)
    if _load().orc_bob_message(d, y.shape[0], _ptr(y), _ptr(bits), _ptr(m)):
        raise ValueError("bad dimension or length")
    return m


def llr(x: np.ndarray, m: np.ndarray, snr: float, d: int = 8) -> np.ndarray:
    """Alice's channel LLRs Q = 2R/sigma_N^2 with R = M X^{-1}."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    q = np.zeros_like(x)
    if _load().orc_llr(d, x.shape[0], _ptr(x), _ptr(m), float(snr), _ptr(q)):
        raise ValueError("bad dimension, length or snr")
    return q


def phi(x: float) -> float:
    """Phi(x) = -ln tanh(x/2)."""
    return _load().orc_phi(float(x))


def decode(code: Code, q: np.ndarray, syn: np.ndarray, max_iter: int,
           et_start: int = 1, clip: float = CLIP, xmin: float = XMIN):
    """Sum-product decoding of one frame (Algorithm 1, syndrome form).

    Returns ``(post, chat, iters, converged)``: FP64 posteriors of every
    variable node, hard decisions, the stopping iteration, and whether
    H chat = syn.
    """
    q = np.ascontiguousarray(q, dtype=np.float64)
    syn = np.ascontiguousarray(syn, dtype=np.uint8)
    assert q.shape == (code.n,) and syn.shape == (code.m,)
    post = np.zeros(code.n, dtype=np.float64)
    chat = np.zeros(code.n, dtype=np.uint8)
    iters = np.zeros(1, dtype=np.int32)
    conv = np.zeros(1, dtype=np.int32)
    rc = _load().orc_decode(code.n, code.m, code.n_edges, _ptr(code.edge_cn),
                            _ptr(code.edge_vn), _ptr(q), _ptr(syn),
                            int(max_iter), int(et_start), float(clip),
                            float(xmin), _ptr(post), _ptr(chat), _ptr(iters),
                            _ptr(conv))
    if rc != 0:
        raise MemoryError("oracle decode: allocation failed")
    return post, chat, int(iters[0]), bool(conv[0])


def row_layers(code: Code, n_groups: int) -> np.ndarray:
    """Layer of every check when the base rows are split into n_groups
    contiguous groups in natural order: base row r (checks r*Z .. r*Z+Z-1)
    belongs to group floor(r * n_groups / mb)."""
    rows = np.arange(code.m, dtype=np.int64) // code.Z
    return (rows * n_groups // code.mb).astype(np.int32)


def decode_layered(code: Code, q: np.ndarray, syn: np.ndarray, max_iter: int,
                   layer: np.ndarray, et_start: int = 1, clip: float = CLIP,
                   xmin: float = XMIN):
    """Layered sum-product decoding of one frame (an extension of Algorithm
    1: checks split into layers visited in order, see orc_decode_layered).
    ``layer[c]`` is the layer of check c. Returns ``(post, chat, iters,
    converged)`` like ``decode``."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    syn = np.ascontiguousarray(syn, dtype=np.uint8)
    layer = np.ascontiguousarray(layer, dtype=np.int32)
    assert q.shape == (code.n,) and syn.shape == (code.m,) and layer.shape == (code.m,)
    n_layers = int(layer.max()) + 1 if code.m else 1
    post = np.zeros(code.n, dtype=np.float64)
    chat = np.zeros(code.n, dtype=np.uint8)
    iters = np.zeros(1, dtype=np.int32)
    conv = np.zeros(1, dtype=np.int32)
    rc = _load().orc_decode_layered(code.n, code.m, code.n_edges, _ptr(code.edge_cn),
                                    _ptr(code.edge_vn), _ptr(q), _ptr(syn), n_layers,
                                    _ptr(layer), int(max_iter), int(et_start), float(clip),
                                    float(xmin), _ptr(post), _ptr(chat), _ptr(iters),
                                    _ptr(conv))
    if rc != 0:
        raise ValueError("oracle layered decode: bad layer ids or allocation failure")
    return post, chat, int(iters[0]), bool(conv[0])
