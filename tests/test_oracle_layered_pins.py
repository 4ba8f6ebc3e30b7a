"""Pins of the oracle's layered schedule (CPU).

The layered schedule is an extension: the paper decodes with flooding
(Algorithm 1). Layered decoding visits the checks layer by layer; the
messages of a layer are computed from the messages as they stand when the
layer starts. The pins below fix it without comparing it to itself:

* one layer is flooding, bit for bit (same sums in the same order);
* on cycle-free graphs it converges to the exact bitwise MAP (brute force);
* on a chain whose checks are visited from one end to the other, one
  iteration already carries every channel LLR to the far end, so the last
  variable's posterior is its exact MAP value after a single iteration,
  where flooding is not (this fails if layers were not committed in order);
* the syndrome sign enters only through (-1)^{s_c} (exact symmetry).
"""
import numpy as np
import pytest

import oracle
from oracle import brute
import synth

from test_oracle_pins import _lift, _random_tree_code


def _frame(code, snr, seed):
    x, y, bits = synth.channel_frame(code.n, snr, seed=seed)
    q = oracle.llr(x, oracle.bob_message(y, bits), snr)
    return q, oracle.syndrome(code, bits), bits


@pytest.mark.parametrize("iters, et_start", [(1, 99), (7, 99), (40, 1)])
def test_one_layer_is_flooding_bit_for_bit(iters, et_start):
    code = oracle.Code.from_dict(synth.rate002_code(24))
    q, syn, _ = _frame(code, 0.3, seed=21)
    ref = oracle.decode(code, q, syn, iters, et_start=et_start)
    got = oracle.decode_layered(code, q, syn, iters, np.zeros(code.m, np.int32),
                                et_start=et_start)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    assert got[2:] == ref[2:]


@pytest.mark.parametrize("seed", range(6))
def test_layered_is_exact_map_on_trees(seed):
    """Cycle-free graphs, random layer assignment, exact mode (no clip)."""
    rng = np.random.default_rng(300 + seed)
    base = _random_tree_code(int(rng.integers(5, 11)), rng)
    d = base if seed % 2 == 0 else _lift(base, 2, rng)
    code = oracle.Code.from_dict(d)
    if code.n > 20:
        pytest.skip("too large for brute force")
    q = rng.standard_normal(code.n) * 1.5 + 0.3
    syn = rng.integers(0, 2, code.m).astype(np.uint8)
    layer = rng.integers(0, 3, code.m).astype(np.int32)
    layer[0] = 2  # three layers in use whatever the draw
    layer[-1] = 0
    iters = code.n + code.m
    post, _, it, _ = oracle.decode_layered(code, q, syn, iters, layer, et_start=iters + 1,
                                           clip=0.0, xmin=1e-300)
    np.testing.assert_allclose(post, brute.bitwise_map_llr(code.dense(), syn, q),
                               rtol=1e-9, atol=1e-9)
    assert it == iters


def test_ordered_layers_carry_a_chain_end_to_end_in_one_iteration():
    """Chain v0 - c0 - v1 - c1 - ... - c(K-1) - vK, check k in layer k."""
    K = 7
    rows = np.repeat(np.arange(K), 2)
    cols = np.stack([np.arange(K), np.arange(1, K + 1)], 1).reshape(-1)
    d = {"mb": K, "nb": K + 1, "Z": 1, "row": rows, "col": cols,
         "shift": np.zeros(2 * K, dtype=int)}
    code = oracle.Code.from_dict(d)
    rng = np.random.default_rng(8)
    q = rng.standard_normal(code.n) * 1.2
    syn = rng.integers(0, 2, code.m).astype(np.uint8)
    ref = brute.bitwise_map_llr(code.dense(), syn, q)
    layer = np.arange(K, dtype=np.int32)
    lay, _, _, _ = oracle.decode_layered(code, q, syn, 1, layer, et_start=2, clip=0.0,
                                         xmin=1e-300)
    flo, _, _, _ = oracle.decode(code, q, syn, 1, et_start=2, clip=0.0, xmin=1e-300)
    assert abs(lay[K] - ref[K]) < 1e-9 * max(1.0, abs(ref[K]))
    assert abs(flo[K] - ref[K]) > 1e-3  # flooding has heard only from v(K-1)
    # the reverse visiting order reaches v0 instead
    rev, _, _, _ = oracle.decode_layered(code, q, syn, 1, layer[::-1].copy(), et_start=2,
                                         clip=0.0, xmin=1e-300)
    assert abs(rev[0] - ref[0]) < 1e-9 * max(1.0, abs(ref[0]))


def test_layered_syndrome_sign_symmetry_is_exact():
    code = oracle.Code.from_dict(synth.rate002_code(16))
    q, syn, bits = _frame(code, 0.5, seed=5)
    layer = oracle.row_layers(code, 7)
    sgn = 1.0 - 2.0 * bits
    p1, c1, i1, v1 = oracle.decode_layered(code, q, syn, 12, layer, et_start=99)
    p0, c0, i0, v0 = oracle.decode_layered(code, q * sgn, np.zeros(code.m, np.uint8), 12,
                                           layer, et_start=99)
    np.testing.assert_array_equal(p1, p0 * sgn)
    np.testing.assert_array_equal(c1, c0 ^ bits)
    assert (i1, v1) == (i0, v0)


def test_row_layers_split_base_rows_in_order():
    code = oracle.Code.from_dict(synth.rate002_code(4))
    lay = oracle.row_layers(code, 7)
    assert lay.shape == (code.m,) and lay.min() == 0 and lay.max() == 6
    rows = np.arange(code.m) // code.Z
    assert np.all(np.diff(lay) >= 0)                      # contiguous groups
    assert all(len(set(lay[rows == r])) == 1 for r in range(code.mb))  # a row is one layer
    np.testing.assert_array_equal(oracle.row_layers(code, 1), 0)
    np.testing.assert_array_equal(oracle.row_layers(code, code.mb), rows)


def test_layered_converges_in_fewer_iterations_than_flooding():
    """Loopy rate-0.02 code at an SNR where both converge: a row-layered
    sweep needs fewer iterations on every frame tried (the reason to layer)."""
    code = oracle.Code.from_dict(synth.rate002_code(64))
    layer = oracle.row_layers(code, code.mb)
    fewer = 0
    for seed in range(4):
        q, syn, _ = _frame(code, 0.6, seed=60 + seed)
        _, _, it_f, cf = oracle.decode(code, q, syn, 60)
        _, _, it_l, cl = oracle.decode_layered(code, q, syn, 60, layer)
        assert cf and cl
        fewer += it_l < it_f
        assert it_l <= it_f
    assert fewer >= 2
