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


def _frames(code_dict, snr, F, seed0, with_oracle_inputs=False):
    fr = make_frames(code_dict, snr, F, seed0=seed0)
    n = fr.code.n
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(torch.from_numpy(fr.x32.reshape(-1)).cuda(),
                    torch.from_numpy(fr.m32.reshape(-1)).cuda(), F * n, snr, llr)
    syn = torch.from_numpy(synth.pack_bits(fr.syn).view(np.int32)).cuda()
    out = [(llr[f * n:(f + 1) * n], syn[f]) for f in range(F)]
    return (out, fr) if with_oracle_inputs else out


def _alone(code, llr, syn, max_iter, params=None):
    dec = q.Decoder(code, 1, params)
    dec.decode(llr, syn, max_iter)
    torch.cuda.synchronize()
    return dec.keys.cpu(), int(dec.converged[0]), int(dec.iters[0])


MIX = {"r002": (synth.rate002_code, 64, 0.08), "r005": (synth.rate005_code, 100, 0.2),
       "r010": (synth.rate010_code, 160, 0.35)}


@pytest.mark.parametrize("schedule, fmt", [(0, 0), (1, 0), (0, 1), (0, 2)])
def test_server_results_equal_alone_decoding_for_a_mix_of_codes(schedule, fmt):
    """Flooding, and layered with one row group per base row; FP32, and for
    flooding FP16 and int8 message storage. Every served frame equals its
    one-frame decode with the same options; with FP32 messages it is also
    checked against the FP64 oracle (the flooding or the layered routine):
    the same stop iteration and flag on every frame, and the oracle's key
    bits on every frame that converged."""
    import oracle
    max_iter = 60
    params = q.qcldpc_params_init(schedule=schedule, msg_format=fmt)
    codes, frames, refs = {}, [], {}
    for i, (name, (mk, Z, snr)) in enumerate(MIX.items()):
        d = mk(Z)
        codes[name] = q.create_code_from(d)
        pairs, fr = _frames(d, snr, 7, 7000 + 100 * i, with_oracle_inputs=True)
        for j, (llr, syn) in enumerate(pairs):
            frames.append((name, j, llr, syn))
            if schedule == 0:
                refs[(name, j)] = oracle.decode(fr.code, fr.q64[j], fr.syn[j], max_iter)
            else:
                layers = oracle.row_layers(fr.code, d["mb"])
                refs[(name, j)] = oracle.decode_layered(fr.code, fr.q64[j], fr.syn[j], max_iter, layers)
            refs[(name, j)] = refs[(name, j)] + (fr.code.k,)
    # a budget of four two-slot chunks: requests wait for room, and empty
    # chunks of one code are released for another
    chunk = 2
    budget = 4 * max(q.qcldpc_pool_workspace(c, chunk, params) for c in codes.values())
    srv = serve.Server(codes, max_iter, params, hbm_budget_bytes=budget, chunk_slots=chunk,
                       idle_seconds=0.0, max_chunk_slots=chunk)
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
    assert srv.peak_used <= budget and srv.footprint <= budget
    n_conv = 0
    for name, j, llr, syn in frames:
        keys, conv, iters = _alone(codes[name], llr, syn, max_iter, params)
        r = results[(name, j)]
        assert (r.converged, r.iters) == (conv, iters), (name, j)
        assert torch.equal(r.keys, keys.view(-1)), (name, j)
        _, chat, it_ref, cv_ref, k = refs[(name, j)]
        if fmt != 0:
            n_conv += conv
            continue
        assert (r.converged, r.iters) == (int(cv_ref), it_ref), ("oracle", name, j)
        if cv_ref:
            got = synth.unpack_bits(r.keys.numpy().view(np.uint32)[None, :], k)[0]
            np.testing.assert_array_equal(got, chat[:k], f"oracle keys {name} {j}")
        n_conv += conv
    assert 0 < n_conv and (schedule == 1 or n_conv < len(frames))


def test_server_moves_memory_between_codes():
    """With a budget of one chunk, a request of another code is admitted by
    releasing the empty chunk of the first code (per-request admission
    against one shared budget), and a request waits while the budget is
    held by running frames."""
    max_iter = 40
    params = q.qcldpc_params_init()
    da, db = synth.rate002_code(64), synth.rate010_code(160)
    codes = {"a": q.create_code_from(da), "b": q.create_code_from(db)}
    fa = _frames(da, 0.08, 2, 8100)
    fb = _frames(db, 0.35, 2, 8200)
    budget = max(q.qcldpc_pool_workspace(c, 2, params) for c in codes.values())
    srv = serve.Server(codes, max_iter, params, hbm_budget_bytes=budget, chunk_slots=2,
                       idle_seconds=1e9, max_chunk_slots=2)
    for j, (llr, syn) in enumerate(fa):
        srv.submit(serve.Request("a", llr, syn, tag=("a", j)))
    srv.submit(serve.Request("b", fb[0][0], fb[0][1], tag=("b", 0)))
    out = srv.tick(passes=1)
    # code a took the only chunk; the b request waits
    assert srv.slots() == {"a": 2, "b": 0} and len(srv.queue) == 1
    res = {r.tag: r for r in out}
    while len(res) < 2:
        res.update({r.tag: r for r in srv.tick(passes=4)})
    srv.submit(serve.Request("b", fb[1][0], fb[1][1], tag=("b", 1)))
    res.update({r.tag: r for r in srv.drain(passes=4)})
    assert srv.slots() == {"a": 0, "b": 2}
    assert srv.peak_used <= budget
    for name, fr in (("a", fa), ("b", fb)):
        for j, (llr, syn) in enumerate(fr):
            keys, conv, iters = _alone(codes[name], llr, syn, max_iter, params)
            r = res[(name, j)]
            assert (r.converged, r.iters) == (conv, iters)
            assert torch.equal(r.keys, keys.view(-1))


def test_server_grows_a_busy_code_in_doubling_chunks():
    """A code whose requests outnumber its slots grows by chunks of 2, 4 and
    8 slots (doubling), and every frame decodes as it would alone."""
    max_iter = 30
    params = q.qcldpc_params_init()
    d = synth.rate002_code(64)
    code = q.create_code_from(d)
    frames = _frames(d, 0.08, 14, 8300)
    srv = serve.Server({"a": code}, max_iter, params, chunk_slots=2, max_chunk_slots=8)
    for j, (llr, syn) in enumerate(frames):
        srv.submit(serve.Request("a", llr, syn, tag=j))
    res = {r.tag: r for r in srv.tick(passes=1)}
    assert sorted(ch.n_slots for ch in srv.chunks["a"]) == [2, 4, 8]
    res.update({r.tag: r for r in srv.drain(passes=4)})
    for j, (llr, syn) in enumerate(frames):
        keys, conv, iters = _alone(code, llr, syn, max_iter, params)
        assert (res[j].converged, res[j].iters) == (conv, iters)
        assert torch.equal(res[j].keys, keys.view(-1))


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
