"""Host-side helpers of the bench studies (no GPU): device bit packing equals
the generator's packing, the paired FER difference, the mix split and the
Poisson trace."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
bench_studies = pytest.importorskip("bench_studies")


def test_pack_dev_matches_synth_pack_bits():
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2, (3, 96)).astype(np.int32)
    bits[:, 31] = 1  # the sign bit of a word
    got = bench_studies.pack_dev(torch.from_numpy(bits)).numpy().view(np.uint32)
    np.testing.assert_array_equal(got, synth.pack_bits(bits.astype(np.uint8)))


def test_paired_difference_counts_discordant_frames():
    ref = np.array([0, 0, 1, 1, 0, 1])
    e = np.array([1, 0, 0, 1, 0, 1])
    p = bench_studies.paired(ref, e)
    assert (p["only_this_fails"], p["only_ref_fails"]) == (1, 1)
    assert p["diff"] == 0.0
    lo, hi = p["diff_ci95"]
    assert lo < 0 < hi
    same = bench_studies.paired(ref, ref)
    assert same["diff_ci95"] == [0.0, 0.0]


def test_split_mix_and_trace():
    counts = bench_studies.split_mix(256)
    assert sum(counts.values()) == 256 and len(counts) == 9
    assert min(counts.values()) >= 10  # every code of the mix is present
    ns = {mk(Z)["nb"] * Z for _, mk, Z, _ in bench_studies.MIX}
    assert ns == {100000, 400000, 1000000}
    tr = bench_studies.trace(np.random.default_rng(0), 100.0, 200, 32, ["a", "b", "c"])
    t = np.array([x[0] for x in tr])
    assert len(tr) == 200 and np.all(np.diff(t) > 0)
    assert {x[1] for x in tr} == {"a", "b", "c"}
    assert all(0 <= x[2] < 32 for x in tr)
    # mean inter-arrival time of a rate-100/s Poisson process
    assert abs(np.diff(t).mean() - 0.01) < 0.003
