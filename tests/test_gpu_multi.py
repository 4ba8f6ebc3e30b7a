"""Batched decoding of several codes in one graph launch (qcldpc_decode_multi)
against one qcldpc_decode call per code and against the FP64 oracle.

Every frame keeps its own stop test inside the shared device loop, so the
key bits, flags and stop iterations must equal the one-code decodes bit for
bit, for every storage format; against the oracle the flags and iterations
are equal on every frame and the key bits on every converged frame
(the bar of test_gpu_parity)."""
import numpy as np
import pytest

import oracle
import synth
from frames import make_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1702_07740_gb300 import qcldpc as q  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    q.load()


def _inputs(fr):
    F, n = fr.F, fr.code.n
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(torch.from_numpy(fr.x32.reshape(-1)).cuda(),
                    torch.from_numpy(fr.m32.reshape(-1)).cuda(), F * n, fr.snr, llr)
    syn = torch.from_numpy(synth.pack_bits(fr.syn).view(np.int32).reshape(-1)).cuda()
    return llr, syn


def _unpack(keys, F, k):
    wk = (k + 31) // 32
    return synth.unpack_bits(keys.cpu().numpy().view(np.uint32)[: F * wk].reshape(F, wk), k)


# (code maker, Z, SNR, frames): rates 0.02, 0.05 and 0.10, ragged frame counts
MIX = [(synth.rate002_code, 64, 0.08, 5), (synth.rate005_code, 100, 0.2, 3),
       (synth.rate010_code, 160, 0.35, 7)]


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_multi_equals_one_decode_per_code_and_the_oracle(fmt):
    max_iter = 60
    params = q.qcldpc_params_init(msg_format=fmt)
    frs, codes, ins = [], [], []
    for i, (mk, Z, snr, F) in enumerate(MIX):
        fr = make_frames(mk(Z), snr, F, seed0=9000 + 100 * i)
        frs.append(fr)
        codes.append(q.create_code_from(fr.code_dict))
        ins.append(_inputs(fr))
    md = q.MultiDecoder(codes, [fr.F for fr in frs], params)
    md.decode([x[0] for x in ins], [x[1] for x in ins], max_iter)
    torch.cuda.synchronize()
    n_conv = 0
    for c, fr in enumerate(frs):
        one = q.Decoder(codes[c], fr.F, params)
        one.decode(ins[c][0], ins[c][1], max_iter)
        torch.cuda.synchronize()
        F = fr.F
        assert torch.equal(md.keys[c][: one.keys.numel()], one.keys), c
        assert torch.equal(md.converged[c][:F], one.converged), c
        assert torch.equal(md.iters[c][:F], one.iters), c
        if fmt != 0:
            continue
        keys = _unpack(md.keys[c], F, fr.code.k)
        conv, its = md.converged[c][:F].cpu().numpy(), md.iters[c][:F].cpu().numpy()
        for f in range(F):
            _, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], max_iter)
            assert (its[f], conv[f]) == (it, int(cv)), (c, f)
            if cv:
                n_conv += 1
                np.testing.assert_array_equal(keys[f], chat[: fr.code.k], f"code {c} frame {f}")
    if fmt == 0:
        assert 0 < n_conv < sum(fr.F for fr in frs)


def test_multi_with_a_repeated_code_and_an_empty_entry():
    """The same code twice (two frame groups with their own workspace parts)
    and a code with no frame."""
    max_iter = 40
    d = synth.rate002_code(64)
    fa = make_frames(d, 0.08, 3, seed0=9500)
    fb = make_frames(d, 0.08, 2, seed0=9600)
    code = q.create_code_from(d)
    other = q.create_code_from(synth.rate010_code(160))
    ia, ib = _inputs(fa), _inputs(fb)
    md = q.MultiDecoder([code, other, code], [3, 0, 2])
    md.decode([ia[0], None, ib[0]], [ia[1], None, ib[1]], max_iter)
    torch.cuda.synchronize()
    for slot, fr, inp in ((0, fa, ia), (2, fb, ib)):
        one = q.Decoder(code, fr.F)
        one.decode(inp[0], inp[1], max_iter)
        torch.cuda.synchronize()
        assert torch.equal(md.keys[slot][: one.keys.numel()], one.keys)
        assert torch.equal(md.iters[slot][: fr.F], one.iters)
        assert torch.equal(md.converged[slot][: fr.F], one.converged)


def test_multi_rejects_bad_arguments():
    code = q.create_code_from(synth.rate002_code(64))
    assert q.qcldpc_decode_multi_workspace([code], [1], q.qcldpc_params_init(msg_format=5)) == 0
    assert q.qcldpc_decode_multi_workspace([code] * 17, [1] * 17) == 0
    md = q.MultiDecoder([code], [1])
    x = torch.zeros(code.n, device="cuda")
    s = torch.zeros((code.m + 31) // 32, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QcldpcError, match="INVAL"):
        q.qcldpc_decode_multi([code], [x], [s], [1], 10, q.qcldpc_params_init(schedule=1), md.keys,
                              md.converged, md.iters, md.workspace, md.ws_bytes)
    with pytest.raises(q.QcldpcError, match="NOMEM"):
        q.qcldpc_decode_multi([code], [x], [s], [1], 10, None, md.keys, md.converged, md.iters,
                              md.workspace, 256)


def test_multi_full_size_matches_one_decode_per_code_and_the_oracle():
    """n = 10^6 frames of the rate-0.02 and rate-0.10 codes in one batched
    decode: bit-identical to one decode per code, and frame 0 of each code
    equal to the oracle's flag and iterations after 20 iterations at a
    converging SNR."""
    from concurrent.futures import ThreadPoolExecutor
    max_iter = 20
    specs = [(synth.rate002_code, 20000, 0.16), (synth.rate010_code, 100000, 1.0)]
    frs, codes, ins = [], [], []
    for i, (mk, Z, snr) in enumerate(specs):
        fr = make_frames(mk(Z), snr, 2, seed0=9700 + 100 * i)
        frs.append(fr)
        codes.append(q.create_code_from(fr.code_dict))
        ins.append(_inputs(fr))
    md = q.MultiDecoder(codes, [2, 2])
    md.decode([x[0] for x in ins], [x[1] for x in ins], max_iter)
    torch.cuda.synchronize()
    for c, fr in enumerate(frs):
        one = q.Decoder(codes[c], 2)
        one.decode(ins[c][0], ins[c][1], max_iter)
        torch.cuda.synchronize()
        assert torch.equal(md.keys[c][: one.keys.numel()], one.keys)
        assert torch.equal(md.iters[c][:2], one.iters) and torch.equal(md.converged[c][:2], one.converged)
    with ThreadPoolExecutor(max_workers=2) as ex:
        refs = list(ex.map(lambda fr: oracle.decode(fr.code, fr.q64[0], fr.syn[0], max_iter), frs))
    for c, (fr, (_, chat, it, cv)) in enumerate(zip(frs, refs)):
        conv, its = int(md.converged[c][0]), int(md.iters[c][0])
        assert (its, conv) == (it, int(cv)), c
        if cv:
            keys = _unpack(md.keys[c], 2, fr.code.k)
            np.testing.assert_array_equal(keys[0], chat[: fr.code.k])


@pytest.mark.parametrize("fmt,layers", [(0, None), (1, None), (2, None), (0, 7), (0, 49)])
def test_frame_groups_equal_one_chain(fmt, layers):
    """A decode whose frames run as side-by-side groups (the default for >= 2
    frames, flooding or layered with `layers` row groups) gives every frame
    the key bits, flag and stop iteration of the one-chain decode: 2, 3 and
    one-frame groups, ragged group sizes, with and without delayed early
    termination."""
    max_iter = 40
    d = synth.rate002_code(64)
    fr = make_frames(d, 0.05, 7, seed0=9800)  # the oracle converges 5 of 7 in 40 iterations
    code = q.create_code_from(fr.code_dict)
    llr, syn = _inputs(fr)
    sched = {} if layers is None else {"schedule": 1, "layers": layers}
    for et in (1, 12):
        ref = q.Decoder(code, fr.F, q.qcldpc_params_init(msg_format=fmt, et_start=et, frame_groups=1, **sched))
        ref.decode(llr, syn, max_iter)
        torch.cuda.synchronize()
        if fmt == 0:
            assert 0 < int(ref.converged.sum()) < fr.F
        for G in (0, 3, 7):
            dec = q.Decoder(code, fr.F, q.qcldpc_params_init(msg_format=fmt, et_start=et, frame_groups=G, **sched))
            dec.decode(llr, syn, max_iter)
            torch.cuda.synchronize()
            assert torch.equal(dec.keys, ref.keys), (et, G)
            assert torch.equal(dec.converged, ref.converged), (et, G)
            assert torch.equal(dec.iters, ref.iters), (et, G)


def test_frame_groups_full_size_equal_one_chain():
    """n = 10^6, 5 frames in the default two groups (3 + 2) against one
    chain, 30 iterations at a converging SNR."""
    max_iter = 30
    fr = make_frames(synth.rate002_code(20000), 0.16, 5, seed0=9900)
    code = q.create_code_from(fr.code_dict)
    llr, syn = _inputs(fr)
    out = []
    for G in (1, 0):
        dec = q.Decoder(code, fr.F, q.qcldpc_params_init(frame_groups=G))
        dec.decode(llr, syn, max_iter)
        torch.cuda.synchronize()
        out.append((dec.keys.clone(), dec.converged.clone(), dec.iters.clone()))
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_frame_groups_rejects_out_of_range():
    code = q.create_code_from(synth.rate002_code(64))
    dec = q.Decoder(code, 2)
    x = torch.zeros(2 * code.n, device="cuda")
    s = torch.zeros(2 * ((code.m + 31) // 32), dtype=torch.int32, device="cuda")
    with pytest.raises(q.QcldpcError, match="INVAL"):
        q.qcldpc_decode(code, x, s, 2, 10, q.qcldpc_params_init(frame_groups=17), dec.keys,
                        dec.converged, dec.iters, dec.workspace, dec.ws_bytes)


def test_frame_groups_edge_iterations_and_graph_reuse():
    """Grouped and one-chain decodes agree at max_iter 0 and 1 (the first
    trip ends every group's loop), and a second decode of other frames
    through the same cached grouped graph equals a fresh one-chain decode
    (each group's state is re-initialised by its own init kernel)."""
    d = synth.rate002_code(64)
    code = q.create_code_from(d)
    fa = make_frames(d, 0.05, 6, seed0=9840)
    fb = make_frames(d, 0.06, 6, seed0=9860)
    ia, ib = _inputs(fa), _inputs(fb)
    grouped = q.Decoder(code, 6)  # default: two groups of 3
    for max_iter in (0, 1, 30):
        ref = q.Decoder(code, 6, q.qcldpc_params_init(frame_groups=1))
        for inp in (ia, ib):
            ref.decode(inp[0], inp[1], max_iter)
            grouped.decode(inp[0], inp[1], max_iter)
            torch.cuda.synchronize()
            assert torch.equal(grouped.keys, ref.keys), max_iter
            assert torch.equal(grouped.converged, ref.converged), max_iter
            assert torch.equal(grouped.iters, ref.iters), max_iter
