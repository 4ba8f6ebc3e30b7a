"""Brute-force references for tiny codes (n <= ~22). TEST INFRASTRUCTURE ONLY.

Enumerates every word x with H x = s and scores it with the channel LLRs
Q_v = ln P(x_v=0)/P(x_v=1), i.e. log-weight w(x) = sum_v (1 - 2 x_v) Q_v / 2
(the BIAWGN channel model of Sec. II-C). From that:

- ``bitwise_map_llr``: exact a-posteriori LLR of every bit over the coset,
  which sum-product decoding (Algorithm 1) reproduces exactly on a cycle-free
  Tanner graph once the messages have crossed the graph;
- ``block_ml``: the most likely word of the coset.

Written with plain numpy integer masks so that it shares nothing with the
C oracle or the CUDA decoder.
"""
from __future__ import annotations

import numpy as np


def _coset_words(H: np.ndarray, s: np.ndarray) -> np.ndarray:
    """All x in {0,1}^n (as uint64 bit masks, bit v = x_v) with H x = s."""
    m, n = H.shape
    if n > 24:
        raise ValueError("brute force limited to n <= 24")
    words = np.arange(1 << n, dtype=np.uint64)
    ok = np.ones(words.shape, dtype=bool)
    for c in range(m):
        mask = np.uint64(0)
        for v in np.nonzero(H[c])[0]:
            mask |= np.uint64(1) << np.uint64(v)
        par = np.bitwise_count(words & mask) & 1
        ok &= par == (int(s[c]) & 1)
    return words[ok]


def _bits_of(words: np.ndarray, n: int) -> np.ndarray:
    shifts = np.arange(n, dtype=np.uint64)
    return ((words[:, None] >> shifts[None, :]) & np.uint64(1)).astype(np.int8)


def _log_weights(bits: np.ndarray, q: np.ndarray) -> np.ndarray:
    return ((1 - 2 * bits.astype(np.float64)) * (q[None, :] / 2.0)).sum(axis=1)


def bitwise_map_llr(H: np.ndarray, s: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Exact posterior LLR ln P(x_v=0 | Q, Hx=s) / P(x_v=1 | Q, Hx=s)."""
    n = H.shape[1]
    words = _coset_words(H, s)
    if words.size == 0:
        raise ValueError("empty coset")
    bits = _bits_of(words, n)
    w = _log_weights(bits, np.asarray(q, dtype=np.float64))
    out = np.empty(n, dtype=np.float64)
    for v in range(n):
        w0 = w[bits[:, v] == 0]
        w1 = w[bits[:, v] == 1]
        l0 = np.logaddexp.reduce(w0) if w0.size else -np.inf
        l1 = np.logaddexp.reduce(w1) if w1.size else -np.inf
        out[v] = l0 - l1
    return out


def block_ml(H: np.ndarray, s: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Most likely word of the coset {x : Hx = s} (0/1 bytes)."""
    n = H.shape[1]
    words = _coset_words(H, s)
    bits = _bits_of(words, n)
    w = _log_weights(bits, np.asarray(q, dtype=np.float64))
    return bits[int(np.argmax(w))].astype(np.uint8)


def gf2_rank(H: np.ndarray) -> int:
    """Rank of a dense 0/1 matrix over GF(2) (Gaussian elimination)."""
    A = (np.asarray(H, dtype=np.uint8) & 1).copy()
    m, n = A.shape
    r = 0
    for c in range(n):
        piv = None
        for i in range(r, m):
            if A[i, c]:
                piv = i
                break
        if piv is None:
            continue
        if piv != r:
            A[[r, piv]] = A[[piv, r]]
        for i in range(m):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        r += 1
        if r == m:
            break
    return r
