"""The psi polynomial constants compiled into the decoder are the ones the
fitting script derives (CPU; no GPU, no library load).

paper_1702_07740_gb300/phi_fit.py fits the two pieces of psi(y) = log2
coth(y ln2 / 2) against mpmath references; csrc/decode_common.cuh carries the
results as FP32 literals. This test reruns the fit and compares every
literal with the fitted value at FP32 precision, so a hand edit of a
constant, or a change of the fit that was not carried into the kernel
source, fails here.
"""
import os
import re

import numpy as np
import pytest

pytest.importorskip("mpmath")

from paper_1702_07740_gb300 import phi_fit  # noqa: E402

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1702_07740_gb300", "csrc", "decode_common.cuh")


def _literals():
    text = open(SRC).read()
    out = {}
    for name, val in re.findall(r"constexpr float (k[CGA]\d?) = ([-+0-9.eE]+)f;", text):
        out[name] = np.float32(float(val))
    return out


def test_kernel_constants_equal_the_fit():
    G, A, C = phi_fit.coefficients()
    lit = _literals()
    want = {"kC": C}
    want.update({f"kG{i}": g for i, g in enumerate(G)})
    want.update({f"kA{i}": a for i, a in enumerate(A)})
    assert set(want) <= set(lit), f"constants missing in the kernel source: {set(want) - set(lit)}"
    for name, v in want.items():
        assert lit[name] == np.float32(v), f"{name}: source {lit[name]!r}, fit {np.float32(v)!r}"


def test_the_two_pieces_reproduce_psi():
    """The fitted pieces, evaluated in FP64 and combined by a max as the
    kernel does, stay within 2e-7 relative of psi from its definition."""
    import mpmath as mpm
    mpm.mp.dps = 30
    G, A, C = (np.asarray(x, dtype=np.float64) for x in phi_fit.coefficients())
    ys = np.concatenate([np.geomspace(1e-6, 1.0, 300), np.linspace(1.0, 40.0, 300)])
    for y in ys:
        w = y * y
        small = C - np.log2(y) + w * (G[0] + w * (G[1] + w * (G[2] + w * G[3])))
        t = 2.0 ** -y
        v = t * t
        large = t * (A[0] + v * (A[1] + v * (A[2] + v * (A[3] + v * A[4]))))
        got = max(small, large)
        u = mpm.mpf(y) * mpm.log(2) / 2
        ref = float(mpm.log(mpm.coth(u)) / mpm.log(2))
        assert abs(got - ref) <= 2e-7 * ref, (y, got, ref)
