"""Layered schedule on the GPU against the oracle's layered mode.

The GPU splits the base rows into G groups (row r in group floor(r G / mb),
oracle.row_layers), computes each group's messages from the state at the
group's start and adds the group's message changes to the posteriors before
the next group. The oracle recomputes every sum from scratch; the GPU keeps
running posteriors, so FP32 rounding accumulates over the updates. The bars
are those of the flooding parity tests: posteriors within 1e-3 max(|L|, 0.1)
after a fixed iteration count, identical flags, iteration counts and key bits
on frames both sides converge on.
"""
import numpy as np
import pytest

import oracle
import synth
from frames import make_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1702_07740_gb300 import qcldpc as q  # noqa: E402
from test_gpu_parity import (assert_posteriors_close, decode_soft, gpu_llr,  # noqa: E402
                             odd_code)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    q.load()


def layered(code, llr, syn, F, iters, groups, **kw):
    return decode_soft(code, llr, syn, F, iters, schedule=1, layers=groups, **kw)


@pytest.mark.parametrize("groups", [0, 7, 1])
def test_layered_fixed_iterations_match_oracle(groups):
    """Z=512, SNR 0.029, 30 iterations without early stop; groups 0 means one
    group per base row (49)."""
    fr = make_frames(synth.rate002_code(512), 0.029, 2)
    code = q.create_code_from(fr.code_dict)
    iters = 30
    keys, conv, its, post = layered(code, gpu_llr(fr), fr.syn, fr.F, iters, groups,
                                    et_start=iters + 1)
    layer = oracle.row_layers(fr.code, groups or fr.code.mb)
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode_layered(fr.code, fr.q64[f], fr.syn[f], iters, layer,
                                                  et_start=iters + 1)
        err = assert_posteriors_close(post[f], ref, f"groups {groups} frame {f}")
        assert its[f] == it == iters and conv[f] == int(cv)
        print(f"groups {groups} frame {f}: max scaled err {err.max():.2e}")


def test_one_group_equals_flooding():
    fr = make_frames(synth.rate002_code(256), 0.1, 2)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    a = layered(code, llr, fr.syn, fr.F, 25, 1, et_start=26)
    b = decode_soft(code, llr, fr.syn, fr.F, 25, et_start=26)
    for f in range(fr.F):
        ref, _, _, _ = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 25, et_start=26)
        assert_posteriors_close(a[3][f], ref, f"one group, frame {f}")
        assert_posteriors_close(b[3][f], ref, f"flooding, frame {f}")


def test_layered_early_stop_matches_oracle():
    fr = make_frames(synth.rate002_code(64), 0.12, 10)
    code = q.create_code_from(fr.code_dict)
    keys, conv, its, post = layered(code, gpu_llr(fr), fr.syn, fr.F, 60, 0)
    layer = oracle.row_layers(fr.code, fr.code.mb)
    n_conv = 0
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode_layered(fr.code, fr.q64[f], fr.syn[f], 60, layer)
        assert (its[f], conv[f]) == (it, int(cv)), f"frame {f}"
        if cv:
            n_conv += 1
            np.testing.assert_array_equal(keys[f], chat[: fr.code.k], f"frame {f}")
            assert_posteriors_close(post[f], ref, f"frame {f}")
    assert n_conv > 0


def test_layered_needs_fewer_iterations_than_flooding():
    fr = make_frames(synth.rate002_code(256), 0.4, 8)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    _, cf, itf, _ = decode_soft(code, llr, fr.syn, fr.F, 80)
    _, cl, itl, _ = layered(code, llr, fr.syn, fr.F, 80, 0)
    both = (cf == 1) & (cl == 1)
    assert both.sum() >= 4
    assert np.all(itl[both] <= itf[both]) and itl[both].sum() < itf[both].sum()


@pytest.mark.parametrize("Z", [5, 37])
def test_layered_ragged_and_irregular_codes(Z):
    d = odd_code(Z)
    fr = make_frames(d, 0.3, 2)
    code = q.create_code_from(d)
    keys, conv, its, post = layered(code, gpu_llr(fr), fr.syn, fr.F, 12, 3, et_start=13)
    layer = oracle.row_layers(fr.code, 3)
    for f in range(fr.F):
        ref, _, _, cv = oracle.decode_layered(fr.code, fr.q64[f], fr.syn[f], 12, layer,
                                              et_start=13)
        assert_posteriors_close(post[f], ref, f"Z={Z} frame {f}")
        assert conv[f] == int(cv)


def test_layered_stream_mode_matches_graph_mode_and_formats_run():
    fr = make_frames(synth.rate002_code(64), 0.12, 4)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    a = layered(code, llr, fr.syn, fr.F, 40, 5)
    b = layered(code, llr, fr.syn, fr.F, 40, 5, launch_mode=1)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    h = layered(code, llr, fr.syn, fr.F, 40, 5, msg_format=1)
    np.testing.assert_array_equal(h[1], a[1])  # FP16 storage: same flags here


def test_layered_full_size_few_iterations():
    """n = 10^6, 16 frames in one launch, one group per base row; frames 0
    and 15 against the oracle after 2 iterations."""
    F, iters = 16, 2
    d = synth.rate002_code(20000)
    first = make_frames(d, 0.029, 1)
    last = make_frames(d, 0.029, 1, seed0=synth.frame_seed(F - 1))
    code = q.create_code_from(d)
    n = first.code.n
    x = np.concatenate([first.x32] + [first.x32 * 0.5] * (F - 2) + [last.x32])
    m = np.concatenate([first.m32] + [first.m32] * (F - 2) + [last.m32])
    syn = np.concatenate([first.syn] + [first.syn] * (F - 2) + [last.syn])
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(torch.from_numpy(x.reshape(-1)).cuda(), torch.from_numpy(m.reshape(-1)).cuda(),
                    F * n, 0.029, llr)
    _, _, _, post = layered(code, llr, syn, F, iters, 0, et_start=iters + 1)
    layer = oracle.row_layers(first.code, first.code.mb)
    for f, fr in ((0, first), (F - 1, last)):
        ref, _, _, _ = oracle.decode_layered(fr.code, fr.q64[0], fr.syn[0], iters, layer,
                                             et_start=iters + 1)
        assert_posteriors_close(post[f], ref, f"frame {f}")


def test_layered_rejects_bad_group_counts():
    code = q.create_code_from(synth.rate002_code(64))
    dec = q.Decoder(code, 1)
    x = torch.zeros(code.n, device="cuda")
    s = torch.zeros((code.m + 31) // 32, dtype=torch.int32, device="cuda")
    for bad in (-1, code.mb + 1):
        params = q.qcldpc_params_init(schedule=1, layers=bad)
        ws = q.qcldpc_decode_workspace(code, 1, params)
        buf = torch.empty(ws, dtype=torch.uint8, device="cuda")
        with pytest.raises(q.QcldpcError, match="INVAL"):
            q.qcldpc_decode(code, x, s, 1, 5, params, dec.keys, dec.converged, dec.iters, buf, ws)
    for bad in (-1, code.mb + 1):
        with pytest.raises(q.QcldpcError):
            q.Pool(code, 2, 10, q.qcldpc_params_init(schedule=1, layers=bad))


def test_autotune_picks_the_fastest_measured_schedule():
    fr = make_frames(synth.rate002_code(512), 0.3, 8)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    lay = q.qcldpc_params_init(schedule=1)
    ws_bytes = q.qcldpc_decode_workspace(code, fr.F, lay)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    wk = (code.k + 31) // 32
    keys = torch.empty(fr.F * wk, dtype=torch.int32, device="cuda")
    conv = torch.empty(fr.F, dtype=torch.int32, device="cuda")
    its = torch.empty(fr.F, dtype=torch.int32, device="cuda")
    syn = torch.from_numpy(synth.pack_bits(fr.syn).view(np.int32).reshape(-1)).cuda()
    best, times = q.qcldpc_autotune(code, llr, syn, fr.F, 60, None, keys, conv, its, ws,
                                    ws_bytes, reps=2)
    assert set(times) == set(q.AUTOTUNE_CANDIDATES)  # mb = 49: all four candidates
    assert all(t > 0 for t in times.values())
    fastest = q.AUTOTUNE_CANDIDATES.index(min(times, key=times.get))
    assert (best.schedule, best.layers) == [(0, 0), (1, 2), (1, 7), (1, 49)][fastest]
    print("autotune ms:", {k: round(v, 3) for k, v in times.items()})
    # the chosen options decode like that schedule
    a = decode_soft(code, llr, fr.syn, fr.F, 60, schedule=best.schedule, layers=best.layers)
    layer = oracle.row_layers(fr.code, best.layers) if best.schedule else None
    for f in range(fr.F):
        if layer is None:
            _, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 60)
        else:
            _, chat, it, cv = oracle.decode_layered(fr.code, fr.q64[f], fr.syn[f], 60, layer)
        assert (a[2][f], a[1][f]) == (it, int(cv))
