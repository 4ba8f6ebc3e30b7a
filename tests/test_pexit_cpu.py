"""Pins of the protograph EXIT threshold tool (CPU).

* J against a direct quadrature of the BIAWGN capacity (scipy), and J_inv;
* regular (3,6) and (4,8) ensembles against their exact density-evolution
  thresholds sigma* = 0.8809 and 0.8314 (Richardson and Urbanke); the
  Gaussian approximation is known to be within about 1 % on these;
* no threshold beats the Shannon limit of its rate;
* the seeded codes' base matrices (rates 0.02, 0.05, 0.10).
"""
import numpy as np
import pytest

import synth
from paper_1702_07740_gb300 import pexit
from paper_ensemble import PAPER_CN, PAPER_THRESHOLD, PAPER_VN_BALANCED, PAPER_VN_PRINTED

integrate = pytest.importorskip("scipy.integrate")
optimize = pytest.importorskip("scipy.optimize")


def _capacity_quad(snr):
    s2 = 1.0 / snr

    def integrand(y):
        p = np.exp(-(y - 1) ** 2 / (2 * s2)) / np.sqrt(2 * np.pi * s2)
        return p * np.log2(1 + np.exp(-2 * y / s2))
    v, _ = integrate.quad(integrand, -40 * np.sqrt(s2) + 1, 40 * np.sqrt(s2) + 1, limit=400)
    return 1.0 - v


@pytest.mark.parametrize("snr", [0.03, 0.3, 1.0, 4.0])
def test_J_is_the_biawgn_capacity(snr):
    assert pexit.biawgn_capacity(snr) == pytest.approx(_capacity_quad(snr), abs=2e-6)


def test_J_inverse():
    s = np.array([0.05, 0.5, 1.0, 2.0, 5.0, 10.0])
    np.testing.assert_allclose(pexit.J_inv(pexit.J(s)), s, rtol=1e-4)
    np.testing.assert_allclose(pexit.J_fast(s), pexit.J(s), atol=1e-6)


@pytest.mark.parametrize("B, sigma_de, rtol", [([[3, 3]], 0.8809, 0.005), ([[4, 4]], 0.8314, 0.015)])
def test_regular_ensembles_match_density_evolution(B, sigma_de, rtol):
    th = pexit.threshold(np.array(B))
    assert 1.0 / np.sqrt(th) == pytest.approx(sigma_de, rel=rtol)
    assert not pexit.converges(np.array(B), th * 0.98)
    assert pexit.converges(np.array(B), th * 1.02)


def _shannon_snr(rate):
    return optimize.brentq(lambda s: pexit.biawgn_capacity(s) - rate, 1e-4, 100.0)


@pytest.mark.parametrize("mk, rate", [(synth.rate002_code, 0.02), (synth.rate005_code, 0.05),
                                      (synth.rate010_code, 0.10)])
def test_seeded_code_thresholds_respect_the_shannon_limit(mk, rate):
    B = pexit.base_matrix(mk(8))
    assert pexit.rate(B) == pytest.approx(rate)
    th = pexit.threshold(B, hi=20.0)
    assert th > _shannon_snr(rate)
    print(f"rate {rate}: PEXIT threshold SNR {th:.4f}, Shannon limit {_shannon_snr(rate):.4f}")


def test_base_matrix_counts_circulants():
    B = pexit.base_matrix(synth.rate002_code(8))
    assert B.shape == (49, 50)
    assert B[:, 0].sum() == 60 and B[:, 1].sum() == 59
    assert np.all(B[np.arange(48), np.arange(2, 50)] == 1)


def test_single_type_met_equals_protograph_exit():
    assert pexit.met_threshold([(1.0, (3,))], [(0.5, (6,))]) == pytest.approx(
        pexit.threshold(np.array([[3, 3]])), rel=2e-3)


def test_paper_ensemble_sockets_rate_and_threshold():
    vn, cn = PAPER_VN_BALANCED, PAPER_CN
    for t in range(3):
        v = sum(w * d[t] for w, d in vn)
        c = sum(w * d[t] for w, d in cn)
        assert v == pytest.approx(c), f"edge type {t + 1}"
    assert sum(w * d[0] for w, d in PAPER_VN_PRINTED) != pytest.approx(
        sum(w * d[0] for w, d in cn))  # the printed fractions do not balance
    assert pexit.met_rate(vn, cn) == pytest.approx(0.02)
    th = pexit.met_threshold(vn, cn, lo=0.005, hi=1.0)
    th_printed = pexit.met_threshold(PAPER_VN_PRINTED, cn, lo=0.005, hi=1.0)
    print(f"paper ensemble: EXIT threshold {th:.5f} (balanced reading), "
          f"{th_printed:.5f} (as printed), density evolution {PAPER_THRESHOLD}")
    assert th == pytest.approx(PAPER_THRESHOLD, rel=0.03)
    assert abs(th - PAPER_THRESHOLD) < abs(th_printed - PAPER_THRESHOLD)
    assert th > _shannon_snr(0.02)


def test_paper_ensemble_fixture_is_the_printed_distribution():
    """The cited fixture (Sec. III-B): its rate is 0.02 under both forms; the
    printed heavy fractions leave the type-1 sockets unbalanced and the read
    form balances them; the printed threshold in dB is 0.04 dB off its
    linear value (the linear value is used)."""
    from paper_ensemble import FIXTURE, PAPER_RATE
    for vn in (PAPER_VN_PRINTED, PAPER_VN_BALANCED):
        assert pexit.met_rate(vn, PAPER_CN) == pytest.approx(PAPER_RATE)
    sockets = lambda types, t: sum(w * d[t] for w, d in types)
    assert sockets(PAPER_VN_BALANCED, 0) == pytest.approx(sockets(PAPER_CN, 0)) == pytest.approx(41 / 400)
    assert sockets(PAPER_VN_PRINTED, 0) == pytest.approx(39 / 400)
    assert 10 * np.log10(FIXTURE["threshold_snr"]) == pytest.approx(-15.43, abs=0.005)
    assert FIXTURE["threshold_db_printed"] == -15.47
