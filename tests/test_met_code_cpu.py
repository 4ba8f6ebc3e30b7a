"""The QC code sampled from the paper's rate-0.02 multi-edge distribution
(Sec. III-B, heavy fractions read as 7/400 and 9/400): node types, socket
counts and rate are those of the distribution (CPU)."""
import numpy as np

import oracle
import synth


def test_met_code_has_the_distribution_of_the_paper():
    Z = 3
    d = synth.met_code(Z)
    assert (d["mb"], d["nb"]) == (1568, 1600)
    col = np.bincount(d["col"], minlength=d["nb"])
    row = np.bincount(d["row"], minlength=d["mb"])
    # variable nodes: 28 of degree 2 + 57, 36 of degree 3 + 57, 1536 of degree 1
    assert np.all(col[:28] == 59) and np.all(col[28:64] == 60) and np.all(col[64:] == 1)
    # check nodes: 960 type-2 of (2, 1), 576 of (3, 1), type-1: 15 of 3, 17 of 7
    assert np.all(row[:960] == 3) and np.all(row[960:1536] == 4)
    assert np.all(row[1536:1551] == 3) and np.all(row[1551:] == 7)
    # every type-2 row has its own degree-1 column on the diagonal
    diag = d["col"] >= 64
    np.testing.assert_array_equal(d["col"][diag] - 64, d["row"][diag])
    # type-1 checks see only the heavy nodes; type-1 sockets per heavy node 2 or 3
    t1 = d["row"] >= 1536
    assert np.all(d["col"][t1] < 64)
    per_col_t1 = np.bincount(d["col"][t1], minlength=64)
    assert np.all(per_col_t1[:28] == 2) and np.all(per_col_t1[28:] == 3)
    # shifts distinct within an entry, in range
    key = (d["row"].astype(np.int64) * d["nb"] + d["col"]) * Z + d["shift"]
    assert len(np.unique(key)) == len(key) and d["shift"].max() < Z
    code = oracle.Code.from_dict(d)
    assert code.k == 32 * Z and code.k / code.n == 0.02


def test_met_code_is_seeded():
    a, b = synth.met_code(5), synth.met_code(5)
    for k in ("row", "col", "shift"):
        np.testing.assert_array_equal(a[k], b[k])
    c = synth.met_code(5, seed=2)
    assert not np.array_equal(a["shift"], c["shift"]) or not np.array_equal(a["col"], c["col"])
