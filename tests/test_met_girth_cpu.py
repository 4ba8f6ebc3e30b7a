"""Shift selection without length-4 cycles for the sampled multi-edge code.

In a QC lift, a closed walk of four circulants e1 - e2 - e3 - e4 (e1, e2 in
one base row, e2, e3 in one base column, e3, e4 in one row, e4, e1 in one
column, consecutive circulants distinct) is a length-4 cycle exactly when
s1 - s2 + s3 - s4 = 0 mod Z. The counter below enumerates every such walk
directly on the circulant list; the girth-6 generator must leave none, and
must keep the uniform generator's base structure (same circulants per base
entry).
"""
import numpy as np

import synth


def closed_4walks(d):
    Z = d["Z"]
    rows, cols, sh = (np.asarray(d[k]).tolist() for k in ("row", "col", "shift"))
    by_row, by_col = {}, {}
    for i, (r, c, s) in enumerate(zip(rows, cols, sh)):
        by_row.setdefault(r, []).append((i, c, s))
        by_col.setdefault(c, []).append((i, r, s))
    n = 0
    for i1, (r1, c1, s1) in enumerate(zip(rows, cols, sh)):
        for i2, c2, s2 in by_row[r1]:
            if i2 == i1:
                continue
            for i3, r2, s3 in by_col[c2]:
                if i3 == i2:
                    continue
                for i4, c4, s4 in by_row[r2]:
                    if c4 != c1 or i4 == i3 or i4 == i1:
                        continue
                    n += (s1 - s2 + s3 - s4) % Z == 0
    return n


def _entries(d):
    return sorted(zip(np.asarray(d["row"]).tolist(), np.asarray(d["col"]).tolist()))


def test_counter_finds_a_planted_4_cycle():
    # two rows, two columns, shifts with s1 - s2 + s3 - s4 = 0 (mod 7)
    d = {"Z": 7, "row": [0, 0, 1, 1], "col": [0, 1, 1, 0], "shift": [3, 1, 5, 0]}
    assert closed_4walks(d) == 4  # one cycle, once from each circulant (row step first)
    d["shift"] = [3, 1, 5, 1]
    assert closed_4walks(d) == 0


def test_girth6_code_has_no_4_cycles_and_the_same_base_structure():
    d0 = synth.met_code(625)
    d6 = synth.met_code(625, girth6=True)
    assert _entries(d0) == _entries(d6)
    assert closed_4walks(d6) == 0
    print("closed 4-walks: uniform", closed_4walks(d0), "girth-6", 0)


def test_girth6_keeps_shifts_distinct_within_an_entry():
    d6 = synth.met_code(64, girth6=True)
    seen = {}
    for r, c, s in zip(d6["row"], d6["col"], d6["shift"]):
        seen.setdefault((int(r), int(c)), []).append(int(s))
    assert all(len(v) == len(set(v)) for v in seen.values())
    assert all(0 <= s < 64 for v in seen.values() for s in v)
