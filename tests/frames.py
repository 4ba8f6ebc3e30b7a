"""Seeded test frames: synthetic channel samples (synth) plus the oracle's
Bob-side message, syndrome and FP64 LLRs, all from the CPU oracle."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle
import synth


@dataclass
class Frames:
    code_dict: dict
    code: oracle.Code
    snr: float
    x32: np.ndarray     # [F, n] float32, Alice
    y32: np.ndarray     # [F, n] float32, Bob
    bits: np.ndarray    # [F, n] uint8, Bob's bits
    m32: np.ndarray     # [F, n] float32, Bob's message from the oracle (FP64 -> FP32)
    q64: np.ndarray     # [F, n] float64, oracle LLRs of (x32, m32)
    syn: np.ndarray     # [F, m] uint8, oracle syndromes

    @property
    def F(self):
        return self.x32.shape[0]


def make_frames(code_dict: dict, snr: float, n_frames: int, seed0: int = synth.FRAME_SEED0,
                d: int = 8) -> Frames:
    code = oracle.Code.from_dict(code_dict)
    xs, ys, bs, ms, qs, ss = [], [], [], [], [], []
    for f in range(n_frames):
        x, y, bits = synth.channel_frame(code.n, snr, seed0 + f)
        x32, y32 = x.astype(np.float32), y.astype(np.float32)
        m32 = oracle.bob_message(y, bits, d=d).astype(np.float32)
        q64 = oracle.llr(x32.astype(np.float64), m32.astype(np.float64), snr, d=d)
        xs.append(x32); ys.append(y32); bs.append(bits); ms.append(m32); qs.append(q64)
        ss.append(oracle.syndrome(code, bits))
    return Frames(code_dict, code, snr, np.stack(xs), np.stack(ys), np.stack(bs),
                  np.stack(ms), np.stack(qs), np.stack(ss))
