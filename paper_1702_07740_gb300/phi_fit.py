"""Derive the FP32 polynomial pieces of the check-node function used by the kernels.

The decoder keeps every LLR in base-2 units (y = x log2(e), x the natural
LLR). In those units Phi(x) = -ln tanh(x/2) becomes

    psi(y) = log2(e) Phi(y ln 2) = log2 coth(y ln2 / 2),

and the check-node rule keeps its form: m2 = psi(sum psi(|L2|)). Working in
base 2 lets the hardware ex2/lg2 take their arguments without scaling.
psi is split at y = 1/ln2 (x = 1):

* small y: psi(y) = C - log2(y) + w G(w), w = y^2, C = 1 - log2(ln 2); w G(w)
  is log2(u coth u) with u = y ln2 / 2, an even function fitted by a cubic
  in w;
* large y: psi(y) = (2/ln 2) atanh(t), t = 2^-y, written t A(t^2) with
  A(v) = (2/ln 2) atanh(sqrt v)/sqrt v, fitted by a quartic in v.

The coefficients are near-minimax fits in relative error (Lawson reweighting
of least squares on Chebyshev nodes) against mpmath references of the two
series. Run ``python -m paper_1702_07740_gb300.phi_fit`` to print them; the
values in ``csrc/decode_common.cuh`` come from this script
(tests/test_phi_fit_cpu.py checks that they match). A development-time helper:
the library never imports it.
"""
from __future__ import annotations

import math

import numpy as np

Y_SPLIT = 1.0 / math.log(2.0)


def _fit(fun, lo, hi, deg, n=400, rounds=50):
    k = np.arange(n)
    xs = (lo + hi) / 2 + (hi - lo) / 2 * np.cos(np.pi * (k + 0.5) / n)
    ys = np.array([fun(x) for x in xs])
    V = np.vander(xs, deg + 1, increasing=True)
    W = 1.0 / np.abs(ys)
    w = np.ones(n)
    c = None
    for _ in range(rounds):
        c, *_ = np.linalg.lstsq(V * (W * w)[:, None], ys * W * w, rcond=None)
        err = np.abs(V @ c - ys) * W
        w = w * np.sqrt(err / err.max()) + 1e-12
        w /= w.max()
    return c


def coefficients():
    import mpmath as mpm
    mpm.mp.dps = 40
    ln2 = mpm.log(2)

    def g_over_w(w):  # log2(u coth u) / y^2, u = y ln2 / 2, w = y^2
        if w == 0:
            return float(ln2 ** 2 / 12 / ln2)  # limit: (u^2/3)/ln2 / y^2
        u = mpm.sqrt(mpm.mpf(w)) * ln2 / 2
        return float(mpm.log(u * mpm.coth(u)) / ln2 / w)

    def a_of_v(v):  # (2/ln2) atanh(sqrt v)/sqrt v
        if v == 0:
            return float(2 / ln2)
        r = mpm.sqrt(mpm.mpf(v))
        return float(2 / ln2 * mpm.atanh(r) / r)

    G = _fit(g_over_w, 0.0, Y_SPLIT ** 2, 3)
    A = _fit(a_of_v, 0.0, float(mpm.power(2, -2 * Y_SPLIT)), 4)
    C = float(1 - mpm.log(ln2, 2))
    return np.float32(G), np.float32(A), np.float32(C)


if __name__ == "__main__":
    G, A, C = coefficients()
    print(f"constexpr float kC = {C:.9e}f;")
    for name, arr in (("G", G), ("A", A)):
        for i, c in enumerate(arr):
            print(f"constexpr float k{name}{i} = {c:.9e}f;")
