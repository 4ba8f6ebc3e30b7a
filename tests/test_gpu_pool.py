"""Pools and the continuous-batching server: every frame's result is the same
alone and in the mix (identical key bits, stop iteration and flag), with
frames of three codes (rates 0.02, 0.05, 0.10) arriving at different times and
sharing the same iteration passes."""
import numpy as np
import pytest

import synth
from frames import make_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1702_07740_gb300 import qcldpc as q  # noqa: E402
from paper_1702_07740_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    q.load()


def _frames(code_dict, snr, F, seed0):
    fr = make_frames(code_dict, snr, F, seed0=seed0)
    n = fr.code.n
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(torch.from_numpy(fr.x32.reshape(-1)).cuda(),
                    torch.from_numpy(fr.m32.reshape(-1)).cuda(), F * n, snr, llr)
    syn = torch.from_numpy(synth.pack_bits(fr.syn).view(np.int32)).cuda()
    return [(llr[f * n:(f + 1) * n], syn[f]) for f in range(F)]


def _alone(code, llr, syn, max_iter, params=None):
    dec = q.Decoder(code, 1, params)
    dec.decode(llr, syn, max_iter)
    torch.cuda.synchronize()
    return dec.keys.cpu(), int(dec.converged[0]), int(dec.iters[0])


MIX = {"r002": (synth.rate002_code, 64, 0.08), "r005": (synth.rate005_code, 100, 0.2),
       "r010": (synth.rate010_code, 160, 0.35)}


@pytest.mark.parametrize("schedule", [0, 1])
def test_server_results_equal_alone_decoding_for_a_mix_of_codes(schedule):
    """Flooding, and layered with one row group per base row."""
    max_iter = 60
    params = q.qcldpc_params_init(schedule=schedule)
    codes, frames = {}, []
    for i, (name, (mk, Z, snr)) in enumerate(MIX.items()):
        d = mk(Z)
        codes[name] = q.create_code_from(d)
        for j, (llr, syn) in enumerate(_frames(d, snr, 7, 7000 + 100 * i)):
            frames.append((name, j, llr, syn))
    srv = serve.Server(codes, {"r002": 3, "r005": 2, "r010": 4}, max_iter, params)
    # arrivals spread over ticks: two frames per tick, interleaved codes
    order = sorted(frames, key=lambda t: (t[1], t[0]))
    results = {}
    while order or srv.pending():
        for _ in range(2):
            if order:
                name, j, llr, syn = order.pop(0)
                srv.submit(serve.Request(name, llr, syn, tag=(name, j)))
        for r in srv.tick(passes=3):
            results[r.tag] = r
    assert len(results) == len(frames)
    n_conv = 0
    for name, j, llr, syn in frames:
        keys, conv, iters = _alone(codes[name], llr, syn, max_iter, params)
        r = results[(name, j)]
        assert (r.converged, r.iters) == (conv, iters), (name, j)
        assert torch.equal(r.keys, keys.view(-1)), (name, j)
        n_conv += conv
    assert 0 < n_conv and (schedule == 1 or n_conv < len(frames))


def test_pool_slots_are_reused_and_states_track_frames():
    d = synth.rate002_code(64)
    code = q.create_code_from(d)
    pool = q.Pool(code, 2, 30)
    torch.cuda.synchronize()
    assert pool.state.cpu().tolist() == [0, 0]
    (llr, syn), = _frames(d, 0.3, 1, 9000)
    ids = torch.arange(2, dtype=torch.int32, device="cuda")
    q.qcldpc_pool_load(pool, 1, ids[1:2], llr, syn)
    torch.cuda.synchronize()
    assert pool.state.cpu().tolist() == [0, 1]
    for _ in range(40):
        q.qcldpc_pool_step(pool, 1)
        if int(pool.state[1]) == 2:
            break
    assert pool.state.cpu().tolist() == [0, 2]
    wk = (code.k + 31) // 32
    keys = torch.empty(wk, dtype=torch.int32, device="cuda")
    conv = torch.empty(1, dtype=torch.int32, device="cuda")
    its = torch.empty(1, dtype=torch.int32, device="cuda")
    q.qcldpc_pool_collect(pool, 1, ids[1:2], keys, conv, its)
    torch.cuda.synchronize()
    assert pool.state.cpu().tolist() == [0, 0]
    ak, ac, ai = _alone(code, llr, syn, 30)
    assert (int(conv), int(its)) == (ac, ai)
    assert torch.equal(keys.cpu(), ak.view(-1))


def test_pool_rejects_bad_arguments():
    code = q.create_code_from(synth.rate002_code(64))
    assert q.qcldpc_pool_workspace(code, 0) == 0
    with pytest.raises(q.QcldpcError):
        q.Pool(code, 2, 10, q.qcldpc_params_init(soft_output=1))


@pytest.mark.parametrize("groups", [7, 0])
def test_layered_pool_slots_at_different_iterations_decode_as_alone(groups):
    """Layered schedule in a pool: frames loaded at different times share
    the passes (each slot at its own iteration) and decode to the same key
    bits, flag and stop iteration as the layered decoder on each frame alone;
    slots are reused after collection."""
    d = synth.rate002_code(64)
    code = q.create_code_from(d)
    max_iter = 40
    params = q.qcldpc_params_init(schedule=1, layers=groups)
    frames = _frames(d, 0.12, 6, 9100)
    alone = []
    for llr, syn in frames:
        dec = q.Decoder(code, 1, params)
        dec.decode(llr, syn, max_iter)
        torch.cuda.synchronize()
        alone.append((dec.keys.cpu(), int(dec.converged[0]), int(dec.iters[0])))
    pool = q.Pool(code, 4, max_iter, params)
    ids = torch.arange(4, dtype=torch.int32, device="cuda")
    wk = (code.k + 31) // 32

    def load(slot, f):
        q.qcldpc_pool_load(pool, 1, ids[slot:slot + 1], frames[f][0], frames[f][1])

    def run_until_done(slots):
        for _ in range(max_iter + 2):
            if all(int(pool.state[s]) == 2 for s in slots):
                return
            q.qcldpc_pool_step(pool, 1)
        raise AssertionError("slots did not finish")

    def collect_and_check(slot, f):
        keys = torch.empty(wk, dtype=torch.int32, device="cuda")
        conv = torch.empty(1, dtype=torch.int32, device="cuda")
        its = torch.empty(1, dtype=torch.int32, device="cuda")
        q.qcldpc_pool_collect(pool, 1, ids[slot:slot + 1], keys, conv, its)
        torch.cuda.synchronize()
        ak, ac, ai = alone[f]
        assert (int(conv), int(its)) == (ac, ai), f"frame {f}"
        assert torch.equal(keys.cpu(), ak.view(-1)), f"frame {f}"

    load(0, 0)
    load(1, 1)
    for _ in range(3):
        q.qcldpc_pool_step(pool, 1)
    load(2, 2)
    load(3, 3)
    run_until_done([0, 1, 2, 3])
    for slot, f in enumerate(range(4)):
        collect_and_check(slot, f)
    load(0, 4)
    q.qcldpc_pool_step(pool, 2)
    load(1, 5)
    run_until_done([0, 1])
    collect_and_check(0, 4)
    collect_and_check(1, 5)
    assert sum(a[1] for a in alone) >= 2
