"""Host arithmetic of the delayed early-termination table (no GPU)."""
import numpy as np

from paper_1702_07740_gb300 import et_lut


def test_start_is_a_low_quantile_of_converged_stops():
    iters = np.array([7, 5, 9, 6, 500, 8, 6, 10, 5, 7])
    conv = np.array([1, 1, 1, 1, 0, 1, 1, 1, 1, 1])
    assert et_lut.start_from_iterations(iters, conv, 500, quantile=0.0) == 5
    assert et_lut.start_from_iterations(iters, conv, 500, quantile=0.5) == 7
    # the frame that never converged does not count
    assert et_lut.start_from_iterations(iters, conv, 500, quantile=1.0) == 10


def test_no_converged_sample_tests_only_at_the_end():
    assert et_lut.start_from_iterations([500, 500], [0, 0], 500) == 500
    assert et_lut.start_from_iterations([0], [1], 500) == 1  # converged before iterating


def test_lookup_takes_the_higher_snr_neighbour():
    lut = et_lut.EtLut(max_iter=500, snrs=[0.1, 0.13, 0.16], starts=[40, 8, 4])
    assert lut.et_start_for(0.05) == 40     # below the table: the lowest SNR's start
    assert lut.et_start_for(0.1) == 40
    assert lut.et_start_for(0.15) == 4      # the higher SNR's (earlier) start
    assert lut.et_start_for(0.3) == 4       # above the table: the highest SNR's start
