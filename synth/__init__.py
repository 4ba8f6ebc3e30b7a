"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module draws random numbers and formats data; it holds none of the
reconciliation or decoding arithmetic (no octonion products, no syndromes,
no LLRs). Both the CUDA path and the CPU oracle consume what it returns.

Workload recipe (stand-in for the paper's codes, which are not published):

* ``protograph_code``: a QC multi-edge base matrix of ``mb`` rows and
  ``nb = mb + 1`` columns. The ``n_heavy`` leftmost columns are heavy: each
  gets one circulant in every row plus, in ``extra[j]`` rows drawn without
  replacement, a second circulant with a different shift (``per_row`` > 1
  gives every row that many circulants instead). The remaining columns are
  degree-1 identity blocks on rows 0, 1, ... (shift 0), forming the long
  unshifted diagonal of Sec. III-C. Shifts are uniform in [0, Z).
* ``met_code``: a QC code sampled from the paper's rate-0.02 multi-edge
  degree distribution (Sec. III-B), 1600 base columns, 1568 base rows.
* ``channel_frame``: x ~ N(0,1), z ~ N(0, 1/snr), y = x + z (the virtual
  BIAWGN channel of Sec. II-C) and Bob's uniform bits.

Generator: numpy PCG64. Code seed 1; frame f uses seed 1000 + f.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CODE_SEED = 1
FRAME_SEED0 = 1000


def protograph_code(mb: int = 49, Z: int = 512, n_heavy: int = 2,
                    extra=(11, 10), per_row: int = 1,
                    seed: int = CODE_SEED) -> dict:
    """Circulant list of the seeded multi-edge protograph code.

    Returns a dict with ``mb, nb, Z`` and int32 arrays ``row, col, shift``
    (one entry per circulant, sorted by row, then column).
    """
    nb = mb + 1
    n_deg1 = nb - n_heavy
    if n_deg1 > mb:
        raise ValueError("more degree-1 columns than rows")
    rng = np.random.Generator(np.random.PCG64(seed))
    entries = []  # (row, col, shift)
    for j in range(n_heavy):
        mult = np.full(mb, per_row, dtype=np.int64)
        if per_row == 1 and extra is not None and j < len(extra) and extra[j] > 0:
            rows2 = rng.choice(mb, size=int(extra[j]), replace=False)
            mult[rows2] += 1
        for r in range(mb):
            k = int(mult[r])
            if k > Z:
                raise ValueError("more circulants in one entry than shifts")
            shifts = rng.choice(Z, size=k, replace=False)
            for s in shifts:
                entries.append((r, j, int(s)))
    for d in range(n_deg1):
        entries.append((d, n_heavy + d, 0))
    entries.sort(key=lambda e: (e[0], e[1]))
    arr = np.array(entries, dtype=np.int64).reshape(-1, 3)
    return {
        "mb": mb, "nb": nb, "Z": Z,
        "row": arr[:, 0].astype(np.int32),
        "col": arr[:, 1].astype(np.int32),
        "shift": arr[:, 2].astype(np.int32),
    }


# The paper's rate-0.02 multi-edge distribution (Sec. III-B) in integral form
# on 1600 base columns, the smallest size at which every fraction is whole,
# with the heavy variable-node fractions read as 7/400 and 9/400 so that the
# type-1 sockets balance (41/400 on both sides).
MET_VN = ((28, 2, 57), (36, 3, 57))          # (count, type-1 degree, type-2 degree)
MET_DEG1_VN = 1536                           # x3 (degree-1, type 3)
MET_CN_T1 = ((15, 3), (17, 7))               # (count, type-1 degree)
MET_CN_T2 = ((960, 2), (576, 3))             # (count, type-2 degree), each with one x3


def met_code(Z: int, seed: int = CODE_SEED, girth6: bool = False) -> dict:
    """Circulant list of a QC code sampled from the paper's rate-0.02
    multi-edge degree distribution.

    Base columns 0..63 are the heavy variable nodes (28 with 2 type-1 and 57
    type-2 sockets, then 36 with 3 and 57), columns 64..1599 the degree-1
    nodes. Base rows 0..1535 are the type-2 checks (960 with 2 type-2
    sockets, then 576 with 3), each with its own degree-1 column (row r,
    column 64 + r, shift 0); rows 1536..1567 the type-1 checks (15 of degree
    3, then 17 of degree 7). Within each edge type the sockets are matched by
    a seeded random permutation; sockets that land in the same base entry
    become circulants with distinct shifts. Shifts are uniform in [0, Z);
    with girth6, each heavy circulant (in seeded random order) takes a
    uniform shift among those that close no length-4 cycle of the lifted
    graph with the circulants placed before it (shifts_avoiding_4cycles).
    The key bits (k = 32 Z) are heavy columns 0..31.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_heavy = sum(c for c, _, _ in MET_VN)
    n_t2 = sum(c for c, _ in MET_CN_T2)
    n_t1 = sum(c for c, _ in MET_CN_T1)
    mb, nb = n_t2 + n_t1, n_heavy + MET_DEG1_VN
    assert MET_DEG1_VN == n_t2
    # variable-side sockets per edge type (column per socket)
    v1, v2, col = [], [], 0
    for count, d1, d2 in MET_VN:
        for _ in range(count):
            v1 += [col] * d1
            v2 += [col] * d2
            col += 1
    c2, row = [], 0
    for count, d2 in MET_CN_T2:
        for _ in range(count):
            c2 += [row] * d2
            row += 1
    c1 = []
    for count, d1 in MET_CN_T1:
        for _ in range(count):
            c1 += [row] * d1
            row += 1
    assert len(v1) == len(c1) and len(v2) == len(c2)
    pairs = list(zip(c1, rng.permutation(v1))) + list(zip(c2, rng.permutation(v2)))
    # group sockets by base entry, draw distinct shifts per entry
    entries = {}
    for r, c in pairs:
        entries[(int(r), int(c))] = entries.get((int(r), int(c)), 0) + 1
    if any(k > Z for k in entries.values()):
        raise ValueError("more circulants in one base entry than shifts")
    if girth6:
        out = shifts_avoiding_4cycles(entries, Z, rng)
    else:
        out = []
        for (r, c), k in sorted(entries.items()):
            for s in rng.choice(Z, size=k, replace=False):
                out.append((r, c, int(s)))
    for d in range(MET_DEG1_VN):
        out.append((d, n_heavy + d, 0))
    out.sort(key=lambda e: (e[0], e[1]))
    arr = np.array(out, dtype=np.int64).reshape(-1, 3)
    return {"mb": mb, "nb": nb, "Z": Z,
            "row": arr[:, 0].astype(np.int32), "col": arr[:, 1].astype(np.int32),
            "shift": arr[:, 2].astype(np.int32)}


def shifts_avoiding_4cycles(entries: dict, Z: int, rng) -> list:
    """Shifts for base entries {(row, col): circulant count}, placed one
    circulant at a time in seeded random entry order. In a QC lift a closed
    walk e - e2 - e3 - e4 over circulants (e, e2 in one base row, e2, e3 in
    one base column, e3, e4 in one row, e4, e in one column, consecutive
    circulants distinct) is a length-4 cycle exactly when
    s - s2 + s3 - s4 = 0 mod Z. A new circulant takes a uniform shift among
    those that close no such walk with the circulants already placed and
    differ from its entry's other shifts (uniform among the distinct ones if
    every shift is excluded). Returns [(row, col, shift)]."""
    keys = sorted(entries)
    by_row, by_col, entry = {}, {}, {}
    out = []
    for i in rng.permutation(len(keys)):
        r, c = keys[i]
        for _ in range(entries[(r, c)]):
            mine = entry.get((r, c), [])
            bad = set(mine)
            for c2, s2 in by_row.get(r, ()):
                for r2, s3 in by_col.get(c2, ()):
                    if r2 == r and s3 == s2:
                        continue  # e3 would be e2
                    for s4 in entry.get((r2, c), ()):
                        if c2 == c and r2 == r and s4 == s3:
                            continue  # e4 would be e3
                        bad.add((s2 - s3 + s4) % Z)
            # walks through the new circulant twice, e - e2 - e - e4, with
            # e2 != e4 in the same entry: 2 s = s2 + s4 mod Z
            for a in range(len(mine)):
                for b in range(len(mine)):
                    if a != b:
                        t = (mine[a] + mine[b]) % Z
                        bad.update(x for x in ((t // 2), (t + Z) // 2) if (2 * x - t) % Z == 0)
            free = np.setdiff1d(np.arange(Z), np.fromiter(bad, dtype=np.int64, count=len(bad)))
            if free.size == 0:
                free = np.setdiff1d(np.arange(Z), np.array(mine, dtype=np.int64))
            s = int(rng.choice(free))
            by_row.setdefault(r, []).append((c, s))
            by_col.setdefault(c, []).append((r, s))
            entry.setdefault((r, c), []).append(s)
            out.append((r, c, s))
    return out


def rate002_code(Z: int, seed: int = CODE_SEED) -> dict:
    """Rate 0.02: 49x50 base, two heavy columns of degree 60 and 59."""
    return protograph_code(49, Z, n_heavy=2, extra=(11, 10), seed=seed)


def rate005_code(Z: int, seed: int = CODE_SEED) -> dict:
    """Rate 0.05: 19x20 base, one heavy column with two circulants per row."""
    return protograph_code(19, Z, n_heavy=1, extra=None, per_row=2, seed=seed)


def rate010_code(Z: int, seed: int = CODE_SEED) -> dict:
    """Rate 0.10: 9x10 base, one heavy column with two circulants per row."""
    return protograph_code(9, Z, n_heavy=1, extra=None, per_row=2, seed=seed)


def channel_frame(n: int, snr: float, seed: int):
    """One frame of the virtual BIAWGN channel.

    Returns float64 ``x`` (Alice), ``y = x + z`` (Bob), and uint8 ``bits``
    (Bob's uniform codeword-position bits; in syndrome form they need not
    be a codeword).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal(n)
    z = rng.standard_normal(n) * np.sqrt(1.0 / snr)
    bits = rng.integers(0, 2, size=n, dtype=np.uint8)
    return x, x + z, bits


def frame_seed(f: int) -> int:
    return FRAME_SEED0 + f


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """0/1 bytes -> uint32 words, bit v in word v // 32 at position v % 32."""
    bits = np.asarray(bits, dtype=np.uint8) & 1
    nw = (bits.shape[-1] + 31) // 32
    pad = np.zeros(bits.shape[:-1] + (nw * 32,), dtype=np.uint8)
    pad[..., : bits.shape[-1]] = bits
    w = pad.reshape(bits.shape[:-1] + (nw, 32)).astype(np.uint64)
    words = (w << np.arange(32, dtype=np.uint64)).sum(axis=-1)
    return words.astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """Inverse of ``pack_bits``."""
    words = np.asarray(words, dtype=np.uint32)
    b = (words[..., :, None] >> np.arange(32, dtype=np.uint32)) & 1
    return b.reshape(words.shape[:-1] + (-1,))[..., :n].astype(np.uint8)


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload (code recipe + channel + iteration budget)."""
    name: str
    Z: int
    snr: float
    max_iter: int
    frames: int
    et: bool
    rate: str = "0.02"
    extra: dict = field(default_factory=dict)

    def code(self) -> dict:
        return {"0.02": rate002_code, "0.05": rate005_code,
                "0.10": rate010_code}[self.rate](self.Z)


# Rate 0.02, Z=512 (n = 25,600), SNR 0.029, 50 fixed iterations.
SINGLE_FRAME_Z512 = Workload("rate0.02_n25600_snr0.029_50it", 512, 0.029, 50, 1, False)
# Rate 0.02, Z=20,000 (n = 10^6), SNR 0.029, up to 500 iterations with stop test.
PAPER_SCALE_Z20000 = Workload("rate0.02_n1e6_snr0.029_500it", 20000, 0.029, 500, 16, True)
