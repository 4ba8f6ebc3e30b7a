"""Derive the FP32 polynomial pieces of Phi(x) = -ln tanh(x/2) used by the kernels.

Phi is split at x = 1:

* x <= 1:  Phi(x) = ln(2/x) + ln(u coth u), u = x/2. The second term is an
  even function, written as w * G(w) with w = x^2 and G a cubic.
* x > 1:   Phi(x) = 2 atanh(t), t = e^{-x} <= e^{-1}; 2 atanh(t) = 2 t A(t^2)
  with A(v) = atanh(sqrt v)/sqrt v = 1 + v/3 + v^2/5 + ..., fitted by a quartic.

The coefficients are near-minimax fits in relative error (Lawson reweighting
of least squares on Chebyshev nodes) against high-precision references of the
two series, computed with mpmath. Run ``python -m paper_1702_07740_gb300.phi_fit``
to print them; the values in ``csrc/decode.cu`` come from this script.
A development-time helper: the library never imports it.
"""
from __future__ import annotations

import numpy as np

X_SPLIT = 1.0


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

    def g_over_w(w):
        if w == 0:
            return 1.0 / 12.0
        u = mpm.sqrt(mpm.mpf(w)) / 2
        return float(mpm.log(u * mpm.coth(u)) / w)

    def a_of_v(v):
        if v == 0:
            return 1.0
        r = mpm.sqrt(mpm.mpf(v))
        return float(mpm.atanh(r) / r)

    G = _fit(g_over_w, 0.0, X_SPLIT ** 2, 3)
    A = _fit(a_of_v, 0.0, float(mpm.e ** (-2 * X_SPLIT)), 4)
    return np.float32(G), np.float32(A)


if __name__ == "__main__":
    G, A = coefficients()
    for name, arr in (("G", G), ("A", A)):
        for i, c in enumerate(arr):
            print(f"constexpr float k{name}{i} = {c:.9e}f;")
