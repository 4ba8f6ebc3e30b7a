"""Delayed early termination: a look-up table of the first iteration to test.

Sec. IV-A: the syndrome test H C = s costs work every iteration, so it is
switched on only after the number of iterations frames of that SNR
empirically need. Here the table maps an SNR to ``et_start`` (the decoder's
first tested iteration). It is built by decoding sample frames at each SNR
with the test on from the first iteration and taking a low quantile of the
iterations at which frames converged, so that few frames run past their
convergence point. Frames that never converge need no early test at all.

``build`` decodes on the GPU through the library; ``et_start_for`` is host
arithmetic only.
"""
from __future__ import annotations

import bisect
from dataclasses import dataclass, field

import numpy as np

from . import qcldpc as q


@dataclass
class EtLut:
    """SNR -> et_start for one code and iteration budget."""
    max_iter: int
    snrs: list = field(default_factory=list)    # ascending
    starts: list = field(default_factory=list)  # et_start per SNR

    def et_start_for(self, snr: float) -> int:
        """et_start of the nearest tabulated SNR at or above ``snr``: a higher
        SNR converges in no more iterations, so its start is no later than
        the true one and no frame runs past its convergence point for want
        of a test. Above the table: the highest SNR's start."""
        i = bisect.bisect_left(self.snrs, snr)
        return self.starts[min(i, len(self.starts) - 1)]


def start_from_iterations(iters: np.ndarray, converged: np.ndarray, max_iter: int,
                          quantile: float = 0.05) -> int:
    """et_start from sample decodes run with the test from iteration 1: the
    ``quantile`` of the converged frames' stopping iterations (at least 1);
    max_iter when no sample converged (only the final test is useful)."""
    its = np.asarray(iters)[np.asarray(converged) == 1]
    if its.size == 0:
        return max(1, int(max_iter))
    return max(1, int(np.floor(np.quantile(its, quantile))))


def build(code: q.Code, frames_at: dict, max_iter: int, params: q.qcldpc_params | None = None,
          quantile: float = 0.05) -> EtLut:
    """Decode each SNR's sample frames with the test from iteration 1 and
    tabulate et_start. ``frames_at`` maps SNR -> (llr device tensor, syndrome
    device tensor, number of frames)."""
    base = params if params is not None else q.qcldpc_params_init()
    lut = EtLut(max_iter=max_iter)
    for snr in sorted(frames_at):
        llr, syn, F = frames_at[snr]
        p = q.qcldpc_params_init(msg_format=base.msg_format, schedule=base.schedule,
                                 layers=base.layers, clip=base.clip, phi_floor=base.phi_floor)
        p.et_start = 1
        dec = q.Decoder(code, F, p)
        dec.decode(llr, syn, max_iter)
        lut.snrs.append(float(snr))
        lut.starts.append(start_from_iterations(dec.iters.cpu().numpy(),
                                                dec.converged.cpu().numpy(), max_iter, quantile))
    return lut
