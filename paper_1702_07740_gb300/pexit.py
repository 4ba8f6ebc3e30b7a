"""BP threshold of a protograph (base matrix) on the BIAWGN channel by
protograph EXIT analysis (Liva and Chiani, "Protograph LDPC codes design
based on EXIT analysis", Globecom 2007): the Gaussian approximation of
density evolution in which every message is a consistent Gaussian LLR,
N(s^2/2, s^2), tracked by its mutual information with the bit.

The paper designs its multi-edge codes by full density evolution (Sec. III);
this tool answers the same question, the decoding threshold of an ensemble,
for the base matrices this library decodes (circulant counts per base entry),
to place the measured FER curves of the seeded codes.

SNR convention: x = +-1, y = x + n, n ~ N(0, 1/snr); the channel LLR
2y/sigma^2 is then N(2 snr, 4 snr), i.e. s_ch^2 = 4 snr. Host arithmetic only.
"""
from __future__ import annotations

import numpy as np

# Gauss-Hermite nodes for E over a standard normal
_GH_X, _GH_W = np.polynomial.hermite_e.hermegauss(96)
_GH_W = _GH_W / _GH_W.sum()


def J(s):
    """Mutual information between a bit and a consistent Gaussian LLR of
    standard deviation s: 1 - E[log2(1 + exp(-L))], L ~ N(s^2/2, s^2)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    out = np.empty_like(s)
    for i, si in enumerate(s):
        if si < 1e-8:
            out[i] = 0.0
            continue
        L = si * si / 2.0 + si * _GH_X
        out[i] = 1.0 - np.dot(_GH_W, np.logaddexp(0.0, -L)) / np.log(2.0)
    return np.clip(out, 0.0, 1.0)


# J is increasing; J^-1 by interpolation on a fine table (log-spaced in s)
_S_TAB = np.concatenate([[0.0], np.geomspace(1e-4, 60.0, 6000)])
_J_TAB = J(_S_TAB)
_J_TAB = np.maximum.accumulate(_J_TAB)


def J_fast(s):
    """J by linear interpolation in the table (vectorised; used inside the
    EXIT iterations)."""
    s = np.asarray(s, dtype=np.float64)
    return np.interp(s, _S_TAB, _J_TAB)


def J_inv(i):
    """Inverse of J on [0, 1) (s for a given mutual information)."""
    i = np.clip(np.asarray(i, dtype=np.float64), 0.0, _J_TAB[-1])
    return np.interp(i, _J_TAB, _S_TAB)


def biawgn_capacity(snr: float) -> float:
    """Capacity of the binary-input AWGN channel (bits per use) = J(2 sqrt(snr))."""
    return float(J(2.0 * np.sqrt(snr))[0])


def base_matrix(code: dict) -> np.ndarray:
    """Edge counts b[r, c] of a circulant list (``synth`` code dict)."""
    B = np.zeros((code["mb"], code["nb"]), dtype=np.int64)
    np.add.at(B, (np.asarray(code["row"]), np.asarray(code["col"])), 1)
    return B


def converges(B: np.ndarray, snr: float, max_iter: int = 2000, tol: float = 1e-6) -> bool:
    """Protograph EXIT: does the a-posteriori information of every variable
    node reach 1 at this SNR? Columns with no edge are ignored."""
    B = np.asarray(B, dtype=np.float64)
    mb, nb = B.shape
    E = B > 0
    s_ch2 = 4.0 * snr
    i_cv = np.zeros((mb, nb))  # check -> variable information per edge type
    used = E.any(axis=0)
    for _ in range(max_iter):
        # variable -> check: channel plus every other incoming edge
        a = np.where(E, J_inv(i_cv) ** 2, 0.0)
        tot = (B * a).sum(axis=0) + s_ch2
        i_vc = np.where(E, J_fast(np.sqrt(np.maximum(tot[None, :] - a, 0.0))), 0.0)
        # check -> variable: 1 - J of the other incoming (1 - I) terms
        b = np.where(E, J_inv(1.0 - i_vc) ** 2, 0.0)
        tot_c = (B * b).sum(axis=1)
        i_cv = np.where(E, 1.0 - J_fast(np.sqrt(np.maximum(tot_c[:, None] - b, 0.0))), 0.0)
        app = J_fast(np.sqrt((B * np.where(E, J_inv(i_cv) ** 2, 0.0)).sum(axis=0) + s_ch2))
        if np.all(app[used] > 1.0 - tol):
            return True
    return False


def threshold(B: np.ndarray, lo: float = 1e-3, hi: float = 10.0, rel: float = 1e-3,
              max_iter: int = 2000) -> float:
    """Smallest SNR at which protograph EXIT converges (bisection in log SNR)."""
    if not converges(B, hi, max_iter):
        raise ValueError("does not converge even at the upper SNR bound")
    while hi / lo > 1.0 + rel:
        mid = np.sqrt(lo * hi)
        if converges(B, mid, max_iter):
            hi = mid
        else:
            lo = mid
    return float(hi)


def rate(B: np.ndarray) -> float:
    """Design rate 1 - mb / nb of a full-rank base matrix."""
    return 1.0 - B.shape[0] / B.shape[1]


# ------------------------------------------------------- multi-edge ensembles

def met_converges(vn_types, cn_types, snr: float, max_iter: int = 5000,
                  tol: float = 1e-6) -> bool:
    """EXIT analysis (Gaussian approximation) of a multi-edge-type ensemble.

    ``vn_types`` / ``cn_types``: lists of (fraction, degree vector d), d[t]
    sockets of edge type t (all variable nodes see the channel). Tracks one
    mutual information per edge type and direction; a node type's outgoing
    information on type t averages over the node types in proportion to
    their type-t sockets. Converges when every variable type with sockets
    reaches a-posteriori information 1."""
    T = len(vn_types[0][1])
    vw = np.array([w for w, _ in vn_types], dtype=np.float64)
    vd = np.array([d for _, d in vn_types], dtype=np.float64)
    cw = np.array([w for w, _ in cn_types], dtype=np.float64)
    cd = np.array([d for _, d in cn_types], dtype=np.float64)
    v_edges = (vw[:, None] * vd).sum(axis=0)   # sockets per type, variable side
    c_edges = (cw[:, None] * cd).sum(axis=0)
    s_ch2 = 4.0 * snr
    i_cv = np.zeros(T)                          # check -> variable, per type
    for _ in range(max_iter):
        a = J_inv(i_cv) ** 2                    # per type
        tot = vd @ a + s_ch2                    # per variable type
        i_vc = np.zeros(T)
        for t in range(T):
            if v_edges[t] <= 0:
                continue
            out = J_fast(np.sqrt(np.maximum(tot - a[t], 0.0)))
            i_vc[t] = np.sum(vw * vd[:, t] * out) / v_edges[t]
        b = J_inv(1.0 - i_vc) ** 2
        tot_c = cd @ b
        for t in range(T):
            if c_edges[t] <= 0:
                continue
            out = 1.0 - J_fast(np.sqrt(np.maximum(tot_c - b[t], 0.0)))
            i_cv[t] = np.sum(cw * cd[:, t] * out) / c_edges[t]
        app = J_fast(np.sqrt(vd @ (J_inv(i_cv) ** 2) + s_ch2))
        if np.all(app > 1.0 - tol):
            return True
    return False


def met_threshold(vn_types, cn_types, lo: float = 1e-3, hi: float = 10.0,
                  rel: float = 1e-3, max_iter: int = 5000) -> float:
    """Smallest SNR at which met_converges holds (bisection in log SNR)."""
    if not met_converges(vn_types, cn_types, hi, max_iter):
        raise ValueError("does not converge even at the upper SNR bound")
    while hi / lo > 1.0 + rel:
        mid = np.sqrt(lo * hi)
        if met_converges(vn_types, cn_types, mid, max_iter):
            hi = mid
        else:
            lo = mid
    return float(hi)


def met_rate(vn_types, cn_types) -> float:
    """Omega(1) - Psi(1) of normalised multi-edge degree distributions."""
    return sum(w for w, _ in vn_types) - sum(w for w, _ in cn_types)
