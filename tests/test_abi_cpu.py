"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every function include/qcldpc.h declares, and validates codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from paper_1702_07740_gb300 import qcldpc as q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "qcldpc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qcldpc_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = q.load()
    declared = _header_functions()
    assert set(declared) == set(q.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_params_defaults():
    p = q.qcldpc_params_init()
    assert p.clip == pytest.approx(15.0)
    assert p.phi_floor == pytest.approx(1e-6)
    assert p.et_start == 1 and p.schedule == 0 and p.msg_format == 0 and p.soft_output == 0
    assert p.layers == 0
    assert (p.cn_threads, p.vn_nodes, p.vn_split) == (0, 0, 0)  # launch shapes: library's choice


def test_code_info_of_the_rate002_protograph():
    d = synth.rate002_code(512)
    code = q.create_code_from(d)
    assert (code.n, code.m, code.k, code.n_edges) == (25600, 25088, 512, 167 * 512)


@pytest.mark.parametrize("bad, status", [
    (dict(shift=[5]), "QCLDPC_E_SHIFT_RANGE"),
    (dict(shift=[-1]), "QCLDPC_E_SHIFT_RANGE"),
    (dict(row=[3]), "QCLDPC_E_INVAL"),
    (dict(col=[9]), "QCLDPC_E_INVAL"),
])
def test_create_code_rejects_bad_entries(bad, status):
    args = dict(row=[0], col=[0], shift=[1])
    args.update(bad)
    with pytest.raises(q.QcldpcError) as ei:
        q.qcldpc_create_code(2, 4, 5, args["row"], args["col"], args["shift"])
    assert status in str(ei.value)


def test_create_code_rejects_duplicate_shift_and_limits():
    with pytest.raises(q.QcldpcError, match="DUP_SHIFT"):
        q.qcldpc_create_code(2, 3, 8, [0, 0], [1, 1], [3, 3])
    with pytest.raises(q.QcldpcError, match="UNSUPPORTED"):
        q.qcldpc_create_code(2, 3, 32, [0] * 17, [0] * 17, list(range(17)))


def test_workspace_size_grows_with_frames_and_soft_output():
    code = q.create_code_from(synth.rate002_code(512))
    w1 = q.qcldpc_decode_workspace(code, 1)
    w16 = q.qcldpc_decode_workspace(code, 16)
    ws = q.qcldpc_decode_workspace(code, 1, q.qcldpc_params_init(soft_output=1))
    assert 0 < w1 < w16 and ws > w1
    # messages of 119 heavy circulants dominate: >= 119 * Z floats per frame
    assert w16 >= 16 * 119 * 512 * 4


def test_layered_workspace_holds_two_message_buffers():
    """The layered schedule keeps the messages of iterations t-1 and t; the
    flooding workspace instead holds the integer posterior accumulators
    (two per heavy node, plus 4096 words of padding)."""
    d = synth.rate002_code(512)
    code = q.create_code_from(d)
    flood = q.qcldpc_decode_workspace(code, 3, q.qcldpc_params_init(frame_groups=1))
    lay = q.qcldpc_decode_workspace(code, 3, q.qcldpc_params_init(schedule=1, frame_groups=1))
    n_h, n_hcols = 119, 2
    acc = -(-4 * (3 * n_hcols * 2 * 512 + 4096) // 256) * 256
    assert lay - flood >= 3 * n_h * 512 * 4 - acc - 256
    assert lay - flood <= 3 * n_h * 512 * 4 - acc + 256


def test_grouped_flooding_workspace_holds_each_group_and_the_whole_batch():
    """Grouped decodes (by default flooding with >= 2 frames; layered when
    frame_groups asks for groups): the workspace holds every group's own
    layout (256-byte aligned, one after the other) and at least one layout
    of the whole batch; one frame, stream launches, soft output, a default
    layered decode or frame_groups = 1 keep one layout; a group count beyond
    16 is invalid."""
    code = q.create_code_from(synth.rate002_code(512))
    align = lambda x: -(-x // 256) * 256
    for sched in (0, 1):
        one = lambda F: q.qcldpc_decode_workspace(code, F, q.qcldpc_params_init(schedule=sched, frame_groups=1))
        for F, G in [(2, 2), (3, 2), (16, 2), (5, 4), (16, 16)]:
            groups = [F // G + (g < F % G) for g in range(G)]
            parts = 0
            for Fg in groups:
                parts = align(parts) + one(Fg)
            p = q.qcldpc_params_init(schedule=sched, frame_groups=G if (G != 2 or sched) else 0)
            got = q.qcldpc_decode_workspace(code, F, p)
            assert got == max(parts, one(F)), (sched, F, G)
            assert got >= one(F)
        assert q.qcldpc_decode_workspace(code, 1, q.qcldpc_params_init(schedule=sched)) == one(1)
    lay1 = q.qcldpc_decode_workspace(code, 6, q.qcldpc_params_init(schedule=1, frame_groups=1))
    assert q.qcldpc_decode_workspace(code, 6, q.qcldpc_params_init(schedule=1)) == lay1
    assert q.qcldpc_decode_workspace(code, 7, q.qcldpc_params_init(frame_groups=9)) == \
        q.qcldpc_decode_workspace(code, 7, q.qcldpc_params_init(frame_groups=7))
    for p in (q.qcldpc_params_init(launch_mode=1), q.qcldpc_params_init(soft_output=1)):
        p1 = q.qcldpc_params_init(launch_mode=p.launch_mode, soft_output=p.soft_output, frame_groups=1)
        assert q.qcldpc_decode_workspace(code, 6, p) == q.qcldpc_decode_workspace(code, 6, p1)
    assert q.qcldpc_decode_workspace(code, 6, q.qcldpc_params_init(frame_groups=17)) == 0
    assert q.qcldpc_decode_workspace(code, 6, q.qcldpc_params_init(frame_groups=-1)) == 0
