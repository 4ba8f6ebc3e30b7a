"""Quantised density evolution (DE) of multi-edge-type LDPC ensembles on the
BIAWGN channel: the exact BP threshold up to grid resolution, where
``pexit`` gives the Gaussian approximation of it.

Sec. III designs the paper's rate-0.02 multi-edge ensemble by density
evolution and states its threshold (0.02863). This module tracks, per edge
type and direction, the full density of the BP message (all-zero codeword,
symmetric channel) on a uniform LLR grid x = k delta, |k| <= K:

* channel: the LLR 2 y snr of y = 1 + n, n ~ N(0, 1/snr), i.e.
  N(2 snr, 4 snr), binned (tails into the end bins);
* variable node: the channel density convolved with the incoming densities
  (one per socket but the outgoing one), computed exactly by FFT and then
  saturated at +-K delta;
* check node: the tanh rule 2 atanh(prod tanh(L/2)) applied pairwise on the
  grid (Richardson and Urbanke's discretised DE): a table R[i, j] of the
  rounded output magnitude for input magnitudes i, j, the output sign the
  product of the input signs. Repeated inputs combine by binary powers.

A type's outgoing density averages the node types in proportion to their
sockets of that type. The ensemble converges at an SNR when every variable
type's a-posteriori error probability falls below ``tol``. Host arithmetic
only (numpy).

SNR convention as in ``pexit``: x = +-1, noise variance 1 / snr.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from math import erf, sqrt


@dataclass
class Grid:
    """Uniform LLR grid x = k delta, k = -K .. K; pmfs are arrays of 2K+1."""
    K: int = 512
    delta: float = 0.05

    def __post_init__(self):
        m = np.arange(self.K + 1) * self.delta
        th = np.tanh(m / 2.0)
        r = 2.0 * np.arctanh(np.clip(np.outer(th, th), 0.0, 1.0 - 1e-16))
        self.R = np.minimum(np.rint(r / self.delta), np.minimum.outer(np.arange(self.K + 1),
                                                                      np.arange(self.K + 1)))
        self.R = self.R.astype(np.int64).ravel()

    @property
    def n(self) -> int:
        return 2 * self.K + 1


def channel_pmf(g: Grid, snr: float) -> np.ndarray:
    """Binned N(2 snr, 4 snr) on the grid, tails in the end bins."""
    mu, sd = 2.0 * snr, 2.0 * sqrt(snr)
    edges = (np.arange(-g.K, g.K + 2) - 0.5) * g.delta
    cdf = np.array([0.5 * (1.0 + erf((e - mu) / (sd * sqrt(2.0)))) for e in edges])
    p = np.diff(cdf)
    p[0] += cdf[0]
    p[-1] += 1.0 - cdf[-1]
    return p / p.sum()


def delta_zero(g: Grid) -> np.ndarray:
    p = np.zeros(g.n)
    p[g.K] = 1.0
    return p


def _clean(p: np.ndarray) -> np.ndarray:
    p = np.maximum(p, 0.0)
    return p / p.sum()


def vn_sum(g: Grid, terms) -> np.ndarray:
    """Density of a sum of independent LLRs: ``terms`` is a list of
    (pmf, multiplicity). Exact convolution by FFT, then saturation."""
    terms = [(p, m) for p, m in terms if m > 0]
    count = sum(m for _, m in terms)
    if count == 0:
        return delta_zero(g)
    full = count * 2 * g.K + 1
    nfft = 1 << int(np.ceil(np.log2(full)))
    F = np.ones(nfft // 2 + 1, dtype=np.complex128)
    for p, m in terms:
        F *= np.fft.rfft(p, nfft) ** m
    s = np.fft.irfft(F, nfft)[:full]
    s = np.maximum(s, 0.0)
    mid = count * g.K
    out = s[mid - g.K: mid + g.K + 1].copy()
    out[0] += s[: mid - g.K].sum()
    out[-1] += s[mid + g.K + 1:].sum()
    return _clean(out)


def _split(g: Grid, p: np.ndarray):
    """(positive, negative) mass by magnitude 0..K; the zero bin is shared."""
    pos = np.empty(g.K + 1)
    neg = np.empty(g.K + 1)
    pos[1:] = p[g.K + 1:]
    neg[1:] = p[g.K - 1:: -1][: g.K]
    pos[0] = neg[0] = 0.5 * p[g.K]
    return pos, neg


def cn_pair(g: Grid, p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Density of 2 atanh(tanh(a/2) tanh(b/2)) for independent a ~ p, b ~ q."""
    ap, an = _split(g, p)
    bp, bn = _split(g, q)
    same = (np.outer(ap, bp) + np.outer(an, bn)).ravel()
    diff = (np.outer(ap, bn) + np.outer(an, bp)).ravel()
    op = np.bincount(g.R, weights=same, minlength=g.K + 1)
    on = np.bincount(g.R, weights=diff, minlength=g.K + 1)
    out = np.zeros(g.n)
    out[g.K + 1:] = op[1:]
    out[: g.K] = on[1:][::-1]
    out[g.K] = op[0] + on[0]
    return _clean(out)


def cn_power(g: Grid, p: np.ndarray, m: int, memo: dict) -> np.ndarray | None:
    """Check-rule combination of m independent copies of p (None for m = 0)."""
    if m <= 0:
        return None
    if m in memo:
        return memo[m]
    if m == 1:
        r = p
    else:
        h = cn_power(g, p, m // 2, memo)
        r = cn_pair(g, h, h)
        if m % 2:
            r = cn_pair(g, r, p)
    memo[m] = r
    return r


def error_probability(g: Grid, p: np.ndarray) -> float:
    return float(p[: g.K].sum() + 0.5 * p[g.K])


def met_de_converges(vn_types, cn_types, snr: float, grid: Grid | None = None,
                     max_iter: int = 2000, tol: float = 1e-7, stall: int = 200,
                     history: list | None = None) -> bool:
    """Discretised DE of a multi-edge ensemble (``pexit.met_converges``
    arguments): does every variable type's a-posteriori error probability
    fall below ``tol`` within ``max_iter`` iterations? A run whose worst
    error probability has not fallen by a relative 1e-6 over ``stall``
    iterations has reached a non-zero fixed point and fails. ``history``,
    if given, receives (iteration, worst error probability) every 5
    iterations."""
    g = grid or Grid()
    T = len(vn_types[0][1])
    vw = np.array([w for w, _ in vn_types], dtype=np.float64)
    vd = np.array([d for _, d in vn_types], dtype=np.int64)
    cw = np.array([w for w, _ in cn_types], dtype=np.float64)
    cd = np.array([d for _, d in cn_types], dtype=np.int64)
    v_edges = (vw[:, None] * vd).sum(axis=0)
    c_edges = (cw[:, None] * cd).sum(axis=0)
    ch = channel_pmf(g, snr)
    c2v = [delta_zero(g) for _ in range(T)]
    hist = []
    for it in range(1, max_iter + 1):
        # variable -> check, per edge type: mixture over variable types
        v2c = []
        for t in range(T):
            if v_edges[t] <= 0:
                v2c.append(delta_zero(g))
                continue
            acc = np.zeros(g.n)
            for w, d in zip(vw, vd):
                if d[t] == 0:
                    continue
                terms = [(ch, 1)] + [(c2v[u], int(d[u] - (u == t))) for u in range(T)]
                acc += w * d[t] * vn_sum(g, terms)
            v2c.append(_clean(acc))
        # check -> variable, per edge type: mixture over check types
        memos = [dict() for _ in range(T)]
        new = []
        for t in range(T):
            if c_edges[t] <= 0:
                new.append(delta_zero(g))
                continue
            acc = np.zeros(g.n)
            for w, d in zip(cw, cd):
                if d[t] == 0:
                    continue
                parts = [cn_power(g, v2c[u], int(d[u] - (u == t)), memos[u]) for u in range(T)]
                parts = [p for p in parts if p is not None]
                r = parts[0] if parts else delta_zero(g)
                for p in parts[1:]:
                    r = cn_pair(g, r, p)
                acc += w * d[t] * r
            new.append(_clean(acc))
        c2v = new
        if it % 5 == 0 or it == max_iter:
            worst = 0.0
            for d in vd:
                post = vn_sum(g, [(ch, 1)] + [(c2v[u], int(d[u])) for u in range(T)])
                worst = max(worst, error_probability(g, post))
            if history is not None:
                history.append((it, worst))
            if worst < tol:
                return True
            # below threshold the error probability settles at a fixed point
            hist.append(worst)
            if len(hist) > stall // 5 and hist[-1] > hist[-1 - stall // 5] * (1.0 - 1e-6):
                return False
    return False


def met_de_threshold(vn_types, cn_types, lo: float, hi: float, rel: float = 2e-3,
                     grid: Grid | None = None, max_iter: int = 2000, tol: float = 1e-7) -> float:
    """Smallest SNR at which ``met_de_converges`` holds (bisection in log
    SNR between lo, which must fail, and hi, which must converge)."""
    g = grid or Grid()
    if not met_de_converges(vn_types, cn_types, hi, g, max_iter, tol):
        raise ValueError("does not converge at the upper SNR bound")
    while hi / lo > 1.0 + rel:
        mid = sqrt(lo * hi)
        if met_de_converges(vn_types, cn_types, mid, g, max_iter, tol):
            hi = mid
        else:
            lo = mid
    return float(hi)
