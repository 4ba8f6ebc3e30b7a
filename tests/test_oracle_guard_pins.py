"""Pins of the oracle's numerical guards (CPU): the message clip and the
Phi-argument floor.

The paper gives no guards (its decoder is FP32, Sec. IV-A); the reading
taken is: every edge message in both directions is clipped to [-clip,
clip], every Phi argument (each |L_vc| and each exclusive sum) is floored at
xmin, and posteriors are not clipped. The tree and MAP pins run with the
guards off, so these cases pin them on their own: each is a one- or
two-check graph worked out by hand, and the expected posteriors below are
written as explicit compositions of Phi(x) = -ln tanh(x/2) (Algorithm 1),
evaluated with 50-digit mpmath, never through the oracle's own Phi.

The worked values show why each case is there:
* Phi(15) = 6.1e-7 lies below the default floor 1e-6, so a degree-2 check
  whose other input is clipped to 15 sends Phi(1e-6) = 14.509, not 15;
* a clipped input 15 instead of 40 shifts a degree-3 check's output by
  ~7e-7, which FP64 resolves easily;
* the output clip matters only when the exclusive sum is empty (a check of
  degree 1) or below Phi(clip): with clipped inputs and degree >= 2 the sum
  is at least Phi(clip), so Phi of it is at most clip.

test_each_planted_guard_mistake_fails_a_pin compiles copies of the oracle
with one guard mistake each and checks that some case here rejects it.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50

CLIP, XMIN = 15.0, 1e-6


def phi(x):
    """Phi(x) = -ln tanh(x / 2), Algorithm 1's check-node function."""
    x = mpmath.mpf(x)
    return -mpmath.log(mpmath.tanh(x / 2))


def _code(checks, n):
    """Z = 1 code with the given checks (lists of variable indices)."""
    rows, cols = [], []
    for r, vs in enumerate(checks):
        for v in vs:
            rows.append(r)
            cols.append(v)
    return oracle.Code(len(checks), n, 1, rows, cols, [0] * len(rows))


def _case_a():
    """One check {v0, v1, v2}, Q = (40, 1, 1), one iteration: the initial
    variable-to-check message of v0 is clipped to 15 (it reaches v1 and v2
    as Phi(15) in their sums) and v0's posterior 40 + m is not clipped."""
    code = _code([[0, 1, 2]], 3)
    q = np.array([40.0, 1.0, 1.0])
    to_v0 = phi(phi(1) + phi(1))
    to_v12 = phi(phi(15) + phi(1))
    exp = [40 + to_v0, 1 + to_v12, 1 + to_v12]
    return code, q, np.zeros(1, np.uint8), 1, CLIP, XMIN, exp


def _case_a_syndrome():
    """Case A with syndrome bit 1: every message of the check changes sign."""
    code, q, _, it, clip, xmin, _ = _case_a()
    to_v0 = phi(phi(1) + phi(1))
    to_v12 = phi(phi(15) + phi(1))
    exp = [40 - to_v0, 1 - to_v12, 1 - to_v12]
    return code, q, np.ones(1, np.uint8), it, clip, xmin, exp


def _case_b():
    """One check {v0, v1}, Q = (40, 3), one iteration: v1 receives
    Phi(max(Phi(15), 1e-6)) = Phi(1e-6), the floor of the exclusive sum."""
    code = _code([[0, 1]], 2)
    q = np.array([40.0, 3.0])
    exp = [40 + phi(phi(3)), 3 + phi(XMIN)]
    return code, q, np.zeros(1, np.uint8), 1, CLIP, XMIN, exp


def _case_c():
    """One check {v0, v1, v2}, Q = (1e-9, 1, -2), one iteration: |L| = 1e-9
    enters the sums as Phi(1e-6) (the floor of a Phi argument); the signs
    follow the product of the other inputs' signs."""
    code = _code([[0, 1, 2]], 3)
    q = np.array([1e-9, 1.0, -2.0])
    exp = [mpmath.mpf(1e-9) - phi(phi(1) + phi(2)),
           1 - phi(phi(XMIN) + phi(2)),
           -2 + phi(phi(XMIN) + phi(1))]
    return code, q, np.zeros(1, np.uint8), 1, CLIP, XMIN, exp


def _case_d():
    """Checks c0 = {v0, v1}, c1 = {v1, v2, v3}, Q = (40, 1, 1, 1), two
    iterations. After iteration 1 v1's message to c1 is 1 + Phi(1e-6) =
    15.509, clipped to 15 in the variable-node step, so in iteration 2 v2
    and v3 receive Phi(Phi(15) + Phi(1)); posteriors are never clipped."""
    code = _code([[0, 1], [1, 2, 3]], 4)
    q = np.array([40.0, 1.0, 1.0, 1.0])
    p = phi(XMIN)                       # c0 -> v1 in both iterations
    a = phi(phi(1) + phi(1))            # c1 -> v1 (both), c1 -> v2, v3 (iteration 1)
    b = phi(phi(15) + phi(1))           # c1 -> v2, v3 in iteration 2
    to_v0 = phi(phi(1 + a))             # c0 -> v0 in iteration 2: v1's extrinsic 1 + a
    exp = [40 + to_v0, 1 + p + a, 1 + b, 1 + b]
    return code, q, np.zeros(2, np.uint8), 2, CLIP, XMIN, exp


def _case_e():
    """One check {v0, v1, v2}, Q = (0, 1, -2): sgn(0) = +1, and |0| is
    floored at 1e-6 inside the sums."""
    code = _code([[0, 1, 2]], 3)
    q = np.array([0.0, 1.0, -2.0])
    exp = [-phi(phi(1) + phi(2)),
           1 - phi(phi(XMIN) + phi(2)),
           -2 + phi(phi(XMIN) + phi(1))]
    return code, q, np.zeros(1, np.uint8), 1, CLIP, XMIN, exp


def _case_f():
    """Checks c0 = {v0} (degree 1) and c1 = {v0, v1}, Q = (1, 2), floor
    1e-9, one iteration. c0's exclusive sum is empty, so its message is
    Phi(max(0, 1e-9)) = 21.42, which the output clip cuts to 15."""
    code = _code([[0], [0, 1]], 2)
    q = np.array([1.0, 2.0])
    exp = [1 + 15 + phi(phi(2)), 2 + phi(phi(1))]
    return code, q, np.zeros(2, np.uint8), 1, CLIP, 1e-9, exp


CASES = {"a": _case_a, "a_syndrome": _case_a_syndrome, "b": _case_b, "c": _case_c,
         "d": _case_d, "e": _case_e, "f": _case_f}


def _check(post, exp):
    exp = np.array([float(e) for e in exp])
    np.testing.assert_allclose(post, exp, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("name", sorted(CASES))
def test_guard_case_flooding(name):
    code, q, syn, iters, clip, xmin, exp = CASES[name]()
    post, _, it, _ = oracle.decode(code, q, syn, iters, et_start=iters + 1, clip=clip, xmin=xmin)
    assert it == iters
    _check(post, exp)


@pytest.mark.parametrize("name", sorted(CASES))
def test_guard_case_layered_one_layer(name):
    """The layered routine with a single layer computes flooding, guards
    included."""
    code, q, syn, iters, clip, xmin, exp = CASES[name]()
    post, _, it, _ = oracle.decode_layered(code, q, syn, iters, np.zeros(code.m, np.int32),
                                           et_start=iters + 1, clip=clip, xmin=xmin)
    assert it == iters
    _check(post, exp)


def test_worked_values():
    """The facts the cases rely on, from the definition of Phi."""
    assert phi(15) < XMIN < phi(14)            # a clipped 15 sits below the floor
    assert abs(phi(phi(15)) - 15) < 1e-30     # Phi is its own inverse
    assert 14.5 < phi(XMIN) < 14.52
    assert phi(1e-9) > 21
    assert 1 + phi(XMIN) > CLIP                # case d: v1 -> c1 is clipped


# ------------------------------------------------- planted mistakes

# Each mutation is (description, text in qcldpc_oracle.c, replacement,
# occurrence): one guard mistake a plausible implementation could make.
# Occurrence 0 is the flooding routine, 1 the layered one.
MUTATIONS = [
    ("initial messages unclipped", "l_vc[e] = clip_msg(q[edge_vn[e]], clip);",
     "l_vc[e] = q[edge_vn[e]];", 0),
    ("variable-node step unclipped (flooding)", "l_vc[e] = clip_msg(ext, clip);", "l_vc[e] = ext;", 0),
    ("variable-node step unclipped (layered)", "l_vc[e] = clip_msg(ext, clip);", "l_vc[e] = ext;", 1),
    ("posteriors clipped (flooding)", "post[v] = total;", "post[v] = clip_msg(total, clip);", 0),
    ("posteriors clipped (layered)", "post[v] = total;", "post[v] = clip_msg(total, clip);", 1),
    ("exclusive-sum floor missing (flooding)", "orc_phi(fmax(sum, xmin)), clip);",
     "orc_phi(sum), clip);", 0),
    ("exclusive-sum floor missing (layered)", "orc_phi(fmax(sum, xmin)), clip);",
     "orc_phi(sum), clip);", 1),
    ("input floor missing (flooding)", "sum += orc_phi(fmax(fabs(l), xmin));",
     "sum += orc_phi(fabs(l));", 0),
    ("input floor missing (layered)", "sum += orc_phi(fmax(fabs(lv), xmin));",
     "sum += orc_phi(fabs(lv));", 0),
    ("output clip missing (flooding)", "m_cv[e] = clip_msg(sign * orc_phi(fmax(sum, xmin)), clip);",
     "m_cv[e] = sign * orc_phi(fmax(sum, xmin));", 0),
    ("output clip missing (layered)", "m_new[e] = clip_msg(sign * orc_phi(fmax(sum, xmin)), clip);",
     "m_new[e] = sign * orc_phi(fmax(sum, xmin));", 0),
    ("floor applied to the output instead of the sum (flooding)",
     "orc_phi(fmax(sum, xmin)), clip);", "fmax(orc_phi(sum), xmin), clip);", 0),
    ("sgn(0) = -1", "return x < 0.0 ? -1.0 : 1.0;", "return x <= 0.0 ? -1.0 : 1.0;", 0),
    ("clip at the wrong level", "if (x > clip)\n        return clip;",
     "if (x > clip)\n        return 0.9 * clip;", 0),
]


def _mutant_lib(tmpdir, text, repl, occurrence):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "qcldpc_oracle.c")).read()
    at = -1
    for _ in range(occurrence + 1):
        at = src.index(text, at + 1)
    mutated = src[:at] + repl + src[at + len(text):]
    c_path = os.path.join(tmpdir, "mutant.c")
    so_path = os.path.join(tmpdir, "mutant.so")
    with open(c_path, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    so_path, c_path, "-lm"], check=True)
    lib = ctypes.CDLL(so_path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.orc_decode.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, i32, dbl, dbl, vp, vp, vp, vp]
    lib.orc_decode.restype = i32
    lib.orc_decode_layered.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp, i32, i32, dbl, dbl,
                                       vp, vp, vp, vp]
    lib.orc_decode_layered.restype = i32
    return lib


def _run(lib, layered, code, q, syn, iters, clip, xmin):
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    q = np.ascontiguousarray(q, dtype=np.float64)
    syn = np.ascontiguousarray(syn, dtype=np.uint8)
    post = np.zeros(code.n)
    chat = np.zeros(code.n, np.uint8)
    it = np.zeros(1, np.int32)
    conv = np.zeros(1, np.int32)
    if layered:
        layer = np.zeros(code.m, np.int32)
        lib.orc_decode_layered(code.n, code.m, code.n_edges, p(code.edge_cn), p(code.edge_vn), p(q),
                               p(syn), 1, p(layer), iters, iters + 1, clip, xmin, p(post), p(chat),
                               p(it), p(conv))
    else:
        lib.orc_decode(code.n, code.m, code.n_edges, p(code.edge_cn), p(code.edge_vn), p(q), p(syn),
                       iters, iters + 1, clip, xmin, p(post), p(chat), p(it), p(conv))
    return post


def _caught(lib):
    for name, make in CASES.items():
        code, q, syn, iters, clip, xmin, exp = make()
        for layered in (False, True):
            try:
                _check(_run(lib, layered, code, q, syn, iters, clip, xmin), exp)
            except AssertionError:
                return True
    return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_each_planted_guard_mistake_fails_a_pin(tmp_path):
    # the unmodified source, through the same loader, passes every case
    os.makedirs(tmp_path / "clean")
    src_dir = os.path.dirname(oracle.__file__)
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    str(tmp_path / "clean" / "clean.so"), os.path.join(src_dir, "qcldpc_oracle.c"),
                    "-lm"], check=True)
    clean = ctypes.CDLL(str(tmp_path / "clean" / "clean.so"))
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    clean.orc_decode.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, i32, dbl, dbl, vp, vp, vp, vp]
    clean.orc_decode_layered.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp, i32, i32, dbl,
                                         dbl, vp, vp, vp, vp]
    assert not _caught(clean)
    missed = []
    for k, (desc, text, repl, occ) in enumerate(MUTATIONS):
        d = tmp_path / f"m{k}"
        os.makedirs(d)
        if not _caught(_mutant_lib(str(d), text, repl, occ)):
            missed.append(desc)
    assert not missed, f"guard mistakes no pin rejects: {missed}"
