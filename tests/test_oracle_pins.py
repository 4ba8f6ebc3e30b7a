"""Pins for the FP64 oracle against facts fixed by the paper and the mathematics.

Nothing here re-types the oracle's own formulas: each check uses an
independent construction (dense circulants from numpy.roll, Hamilton's
quaternion product, brute-force MAP over the coset, exact sign symmetry,
closed forms of the noise-free channel, BIAWGN consistency statistics, the
printed d=2 noise form of Sec. II-C).
"""
import numpy as np
import pytest

import oracle
from oracle import brute
import synth


# ---------------------------------------------------------------- expansion

def _dense_by_roll(code_dict):
    """H from the paper's definition: base value i -> identity shifted right."""
    mb, nb, Z = code_dict["mb"], code_dict["nb"], code_dict["Z"]
    H = np.zeros((mb * Z, nb * Z), dtype=np.uint8)
    eye = np.eye(Z, dtype=np.uint8)
    for r, c, s in zip(code_dict["row"], code_dict["col"], code_dict["shift"]):
        H[r * Z:(r + 1) * Z, c * Z:(c + 1) * Z] ^= np.roll(eye, int(s), axis=1)
    return H


@pytest.mark.parametrize("Z", [1, 2, 3, 5, 8])
def test_expansion_matches_shifted_identities(Z):
    rng = np.random.default_rng(Z)
    mb, nb = 4, 6
    rows, cols, shifts = [], [], []
    for r in range(mb):
        for c in range(nb):
            k = rng.integers(0, min(3, Z) + 1)
            for s in rng.choice(Z, size=k, replace=False):
                rows.append(r); cols.append(c); shifts.append(int(s))
    d = {"mb": mb, "nb": nb, "Z": Z, "row": np.array(rows), "col": np.array(cols),
         "shift": np.array(shifts)}
    code = oracle.Code.from_dict(d)
    H = _dense_by_roll(d)
    np.testing.assert_array_equal(code.dense(), H)
    # row/column weights equal the base weights expanded Z times
    base = np.zeros((mb, nb), dtype=np.int64)
    for r, c in zip(rows, cols):
        base[r, c] += 1
    np.testing.assert_array_equal(H.sum(axis=1), np.repeat(base.sum(axis=1), Z))
    np.testing.assert_array_equal(H.sum(axis=0), np.repeat(base.sum(axis=0), Z))
    assert code.n_edges == len(rows) * Z


def test_expansion_rejects_bad_shift():
    with pytest.raises(ValueError):
        oracle.Code(2, 3, 4, [0], [0], [4])


def test_protograph_recipe_degrees():
    d = synth.rate002_code(64)
    code = oracle.Code.from_dict(d)
    H = code.dense()
    colw = H.sum(axis=0).reshape(50, 64)
    assert (colw[0] == 60).all() and (colw[1] == 59).all()
    assert (colw[2:] == 1).all()
    assert code.k == 64 and code.n == 3200
    # edge count: 119 heavy + 48 identity circulants
    assert code.n_edges == 167 * 64


# ----------------------------------------------------------------- syndrome

def test_syndrome_equals_dense_product_and_is_linear():
    d = synth.rate002_code(16)
    code = oracle.Code.from_dict(d)
    H = _dense_by_roll(d).astype(np.int64)
    rng = np.random.default_rng(7)
    for _ in range(5):
        x = rng.integers(0, 2, code.n).astype(np.uint8)
        y = rng.integers(0, 2, code.n).astype(np.uint8)
        sx, sy = oracle.syndrome(code, x), oracle.syndrome(code, y)
        np.testing.assert_array_equal(sx, (H @ x) % 2)
        np.testing.assert_array_equal(oracle.syndrome(code, x ^ y), sx ^ sy)


# ------------------------------------------------------ Cayley-Dickson algebra

def _hamilton(a, b):
    a0, a1, a2, a3 = a
    b0, b1, b2, b3 = b
    return np.array([
        a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3,
        a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2,
        a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1,
        a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0,
    ])


def test_cd_low_dimensions_are_reals_complex_quaternions():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        assert oracle.cd_mul(a[:1], b[:1])[0] == pytest.approx(a[0] * b[0])
        z = complex(a[0], a[1]) * complex(b[0], b[1])
        np.testing.assert_allclose(oracle.cd_mul(a[:2], b[:2]), [z.real, z.imag], rtol=1e-14)
        np.testing.assert_allclose(oracle.cd_mul(a, b), _hamilton(a, b), rtol=1e-13, atol=1e-14)


def _left_matrix(a):
    d = a.shape[0]
    return np.stack([oracle.cd_mul(a, np.eye(d)[j]) for j in range(d)], axis=1)


def _right_matrix(a):
    d = a.shape[0]
    return np.stack([oracle.cd_mul(np.eye(d)[j], a) for j in range(d)], axis=1)


def _conj(a):
    c = -a.copy()
    c[0] = a[0]
    return c


def test_octonion_norm_alternativity_orthogonality():
    rng = np.random.default_rng(2)
    for _ in range(50):
        a, b = rng.standard_normal(8), rng.standard_normal(8)
        ab = oracle.cd_mul(a, b)
        assert np.linalg.norm(ab) == pytest.approx(np.linalg.norm(a) * np.linalg.norm(b), rel=1e-13)
        # right cancellation used by the paper: (a b) conj(b) = |b|^2 a
        np.testing.assert_allclose(oracle.cd_mul(ab, _conj(b)), (b @ b) * a, rtol=1e-12, atol=1e-12)
        # left alternativity a (a b) = (a a) b
        np.testing.assert_allclose(oracle.cd_mul(a, ab), oracle.cd_mul(oracle.cd_mul(a, a), b),
                                   rtol=1e-12, atol=1e-12)
        La, Ra = _left_matrix(a), _right_matrix(a)
        np.testing.assert_allclose(La.T @ La, (a @ a) * np.eye(8), atol=1e-12)
        np.testing.assert_allclose(Ra.T @ Ra, (a @ a) * np.eye(8), atol=1e-12)


def test_octonion_units_and_nonassociativity():
    E = np.eye(8)
    for i in range(1, 8):
        np.testing.assert_allclose(oracle.cd_mul(E[i], E[i]), -E[0])
        for j in range(1, 8):
            if i != j:
                np.testing.assert_allclose(oracle.cd_mul(E[i], E[j]), -oracle.cd_mul(E[j], E[i]))
                p = oracle.cd_mul(E[i], E[j])
                assert np.count_nonzero(p) == 1 and np.abs(p).max() == 1.0
    # octonions are not associative (quaternions are)
    found = False
    for i in range(1, 8):
        for j in range(1, 8):
            for k in range(1, 8):
                l = oracle.cd_mul(oracle.cd_mul(E[i], E[j]), E[k])
                r = oracle.cd_mul(E[i], oracle.cd_mul(E[j], E[k]))
                if not np.allclose(l, r):
                    found = True
    assert found
    rng = np.random.default_rng(3)
    a, b, c = (rng.standard_normal(4) for _ in range(3))
    np.testing.assert_allclose(oracle.cd_mul(oracle.cd_mul(a, b), c),
                               oracle.cd_mul(a, oracle.cd_mul(b, c)), atol=1e-12)


# ------------------------------------------------------------ 8-D / d-D map

def test_d2_noise_matches_printed_form():
    """Sec. II-C: for the all-zero word, N_1 = a Z_1 + b Z_2, N_2 = a Z_2 - b Z_1
    with a = (X_1+X_2)/|X|^2, b = (X_2-X_1)/|X|^2, variance (a^2+b^2) sigma_Z^2."""
    rng = np.random.default_rng(4)
    snr = 0.25
    n = 2000
    x = rng.standard_normal(n)
    z = rng.standard_normal(n) * np.sqrt(1 / snr)
    bits = np.zeros(n, dtype=np.uint8)
    m = oracle.bob_message(x + z, bits, d=2)
    q = oracle.llr(x, m, snr, d=2)
    X1, X2, Z1, Z2 = x[0::2], x[1::2], z[0::2], z[1::2]
    nrm = X1 ** 2 + X2 ** 2
    sigma_n2 = 2 * (1 / snr) / nrm          # d sigma_Z^2 / |X|^2
    R = q * np.repeat(sigma_n2, 2) / 2.0     # invert Q = 2R / sigma_N^2
    a = (X1 + X2) / nrm
    b = (X2 - X1) / nrm
    np.testing.assert_allclose(R[0::2] - 1.0, a * Z1 + b * Z2, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(R[1::2] - 1.0, a * Z2 - b * Z1, rtol=1e-9, atol=1e-9)
    # the printed variance (a^2+b^2) sigma_Z^2 equals d sigma_Z^2/|X|^2 for d=2
    np.testing.assert_allclose((a ** 2 + b ** 2) / snr, sigma_n2, rtol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 4, 8])
def test_noise_free_channel_gives_scaled_signs(d):
    """With Z = 0, R = U exactly, so Q_j = 2 U_j |X|^2 snr / d."""
    rng = np.random.default_rng(5)
    n = 64 * d
    x = rng.standard_normal(n)
    bits = rng.integers(0, 2, n).astype(np.uint8)
    snr = 0.029
    q = oracle.llr(x, oracle.bob_message(x, bits, d=d), snr, d=d)
    u = 1.0 - 2.0 * bits
    nrm = np.repeat((x.reshape(-1, d) ** 2).sum(axis=1), d)
    np.testing.assert_allclose(q, 2 * u * nrm * snr / d, rtol=1e-12)


def test_8d_llr_is_consistent_biawgn():
    """Given |X|^2, Q U ~ N(mu, 2 mu) with mu = |X|^2 snr / 4 (d = 8), so
    E[Q U] = 2 snr overall. Checked in |X|^2 bins with 6-sigma bounds."""
    snr = 0.5
    n = 8 * 40000
    x, y, bits = synth.channel_frame(n, snr, seed=99)
    q = oracle.llr(x, oracle.bob_message(y, bits), snr)
    qu = q * (1.0 - 2.0 * bits)
    nrm = np.repeat((x.reshape(-1, 8) ** 2).sum(axis=1), 8)
    assert qu.mean() == pytest.approx(2 * snr, rel=0.02)
    edges = np.quantile(nrm, [0.0, 0.2, 0.4, 0.6, 0.8, 1.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (nrm >= lo) & (nrm < hi)
        resid = qu[sel] - nrm[sel] * snr / 4.0
        # standardised residual: zero mean, unit variance
        zres = resid / np.sqrt(2 * nrm[sel] * snr / 4.0)
        k = sel.sum()
        assert abs(zres.mean()) < 6 / np.sqrt(k)
        assert abs(zres.var() - 1.0) < 6 * np.sqrt(2.0 / k)


def test_llr_rejects_bad_length():
    with pytest.raises(ValueError):
        oracle.llr(np.ones(12), np.ones(12), 0.1, d=8)


# ---------------------------------------------------------------------- Phi

def test_phi_involution_and_asymptotes():
    for x in np.geomspace(1e-4, 25, 60):
        assert oracle.phi(oracle.phi(x)) == pytest.approx(x, rel=1e-10)
    for x in [1e-6, 1e-8, 1e-12]:
        assert oracle.phi(x) == pytest.approx(np.log(2 / x), rel=1e-9)
    for x in [20.0, 30.0, 40.0]:
        assert oracle.phi(x) == pytest.approx(2 * np.exp(-x), rel=1e-9)


# ---------------------------------------------------------------- decoding

def _random_tree_code(n_vn, rng):
    """A random cycle-free Tanner graph with every check of degree >= 2.

    Returned as a base matrix with Z = 1 (one circulant per edge)."""
    vns, cns = [0], []
    edges = []
    next_v, next_c = 1, 0
    while next_v < n_vn:
        if cns and rng.random() < 0.6:
            c = cns[rng.integers(len(cns))]
            edges.append((c, next_v)); vns.append(next_v); next_v += 1
        else:
            v = vns[rng.integers(len(vns))]
            edges.append((next_c, v)); cns.append(next_c); next_c += 1
    deg = np.zeros(next_c, dtype=int)
    for c, _ in edges:
        deg[c] += 1
    for c in range(next_c):
        if deg[c] < 2:
            edges.append((c, next_v)); next_v += 1
    mb, nb = next_c, next_v
    edges.sort()
    return {"mb": mb, "nb": nb, "Z": 1,
            "row": np.array([e[0] for e in edges]), "col": np.array([e[1] for e in edges]),
            "shift": np.zeros(len(edges), dtype=int)}


def _lift(base, Z, rng):
    d = dict(base)
    d["Z"] = Z
    d["shift"] = rng.integers(0, Z, len(base["row"]))
    return d


@pytest.mark.parametrize("seed", range(8))
def test_bp_is_exact_map_on_trees(seed):
    """On a cycle-free graph sum-product returns the exact bitwise MAP LLRs
    (exact mode: no clipping, Phi floor far below any message)."""
    rng = np.random.default_rng(100 + seed)
    base = _random_tree_code(int(rng.integers(5, 11)), rng)
    d = base if seed % 2 == 0 else _lift(base, 2, rng)
    code = oracle.Code.from_dict(d)
    if code.n > 20:
        pytest.skip("too large for brute force")
    H = code.dense()
    q = rng.standard_normal(code.n) * 1.5 + 0.3
    syn = rng.integers(0, 2, code.m).astype(np.uint8)
    iters = code.n + code.m
    post, chat, it, conv = oracle.decode(code, q, syn, iters, et_start=iters + 1,
                                         clip=0.0, xmin=1e-300)
    ref = brute.bitwise_map_llr(H, syn, q)
    np.testing.assert_allclose(post, ref, rtol=1e-9, atol=1e-9)
    assert it == iters


def test_syndrome_sign_symmetry_is_exact():
    """Decoding (Q, s = H c) equals decoding ((-1)^c Q, 0) with every
    posterior sign flipped by (-1)^c: the syndrome sign (-1)^{s_c} is the only
    place the two differ. Bit-exact, clipping on, loopy code."""
    d = synth.rate002_code(16)
    code = oracle.Code.from_dict(d)
    x, y, bits = synth.channel_frame(code.n, 0.5, seed=5)
    q = oracle.llr(x, oracle.bob_message(y, bits), 0.5)
    syn = oracle.syndrome(code, bits)
    sgn = 1.0 - 2.0 * bits
    p1, c1, i1, v1 = oracle.decode(code, q, syn, 12, et_start=99)
    p0, c0, i0, v0 = oracle.decode(code, q * sgn, np.zeros(code.m, np.uint8), 12, et_start=99)
    np.testing.assert_array_equal(p1, p0 * sgn)
    np.testing.assert_array_equal(c1, c0 ^ bits)
    assert (i1, v1) == (i0, v0)


def test_zero_iterations_and_stop_rule():
    d = synth.rate002_code(8)
    code = oracle.Code.from_dict(d)
    x, y, bits = synth.channel_frame(code.n, 0.029, seed=3)
    q = oracle.llr(x, oracle.bob_message(y, bits), 0.029)
    syn = oracle.syndrome(code, bits)
    post, chat, it, conv = oracle.decode(code, q, syn, 0)
    np.testing.assert_array_equal(post, q)
    assert it == 0
    assert conv == bool((oracle.syndrome(code, chat) == syn).all())
    # noise-free LLRs of Bob's own bits satisfy the syndrome at the first test
    q_clean = 5.0 * (1.0 - 2.0 * bits)
    post, chat, it, conv = oracle.decode(code, q_clean, syn, 20, et_start=1)
    assert conv and it == 1
    np.testing.assert_array_equal(chat, bits)


def test_loopy_bp_agrees_with_ml_at_high_snr():
    """Small loopy code: at high SNR BP's decision equals the block-ML word on
    most frames, and BP never beats ML at recovering the transmitted word."""
    rng = np.random.default_rng(11)
    d = {"mb": 3, "nb": 6, "Z": 3}
    rows, cols, shifts = [], [], []
    for r in range(3):
        for c in range(6):
            if (r + c) % 3 != 2:
                rows.append(r); cols.append(c); shifts.append(int(rng.integers(3)))
    d.update(row=np.array(rows), col=np.array(cols), shift=np.array(shifts))
    code = oracle.Code.from_dict(d)
    H = code.dense()
    agree = bp_err = ml_err = 0
    frames = 60
    for f in range(frames):
        bits = rng.integers(0, 2, code.n).astype(np.uint8)
        syn = oracle.syndrome(code, bits)
        q = (1 - 2.0 * bits) * 4.0 + rng.standard_normal(code.n) * 2.0
        _, chat, _, _ = oracle.decode(code, q, syn, 30)
        ml = brute.block_ml(H, syn, q)
        agree += int((chat == ml).all())
        bp_err += int((chat != bits).any())
        ml_err += int((ml != bits).any())
    assert agree >= 0.8 * frames
    assert ml_err <= bp_err + 3
