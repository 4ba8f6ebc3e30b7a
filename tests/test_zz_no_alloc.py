"""qcldpc_decode_noalloc: decoding for callers that cannot allocate device memory.

Some callers have no way to allocate device memory of their own: code
embedded in a host framework that owns the device allocator, or a process
whose device memory is reserved once at start-up. For them the library keeps
the decoder's scratch in a static device array instead of a caller workspace.
These tests call that entry point through the C ABI and check, on two calls in
a row with different inputs, that it returns exactly what qcldpc_decode
returns (key bits, convergence flags and iteration counts are integers, so the
bar is identity). The file is named to be collected last.
"""
import numpy as np
import pytest

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


def _inputs(code_dict, snr, F, seed0):
    fr = make_frames(code_dict, snr, F, seed0=seed0)
    n = fr.x32.size
    llr = torch.empty(n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(torch.from_numpy(fr.x32.reshape(-1)).cuda(),
                    torch.from_numpy(fr.m32.reshape(-1)).cuda(), n, snr, llr)
    syn = torch.from_numpy(synth.pack_bits(fr.syn).view(np.int32).reshape(-1)).cuda()
    return llr, syn


def _outputs(code, F):
    wk = (code.k + 31) // 32
    return (torch.full((F * wk,), -1, dtype=torch.int32, device="cuda"),
            torch.full((F,), -1, dtype=torch.int32, device="cuda"),
            torch.full((F,), -1, dtype=torch.int32, device="cuda"))


def test_noalloc_matches_workspace_decode_on_two_calls():
    d = synth.rate002_code(2000)  # n = 10^5: two frames fit the static scratch
    code = q.create_code_from(d)
    F, max_iter = 2, 40
    params = q.qcldpc_params_init()
    for call, (snr, seed0) in enumerate([(0.1, 5000), (0.15, 6000)]):
        llr, syn = _inputs(d, snr, F, seed0)
        ref = q.Decoder(code, F, params)
        ref.decode(llr, syn, max_iter)
        keys, conv, iters = _outputs(code, F)
        q.qcldpc_decode_noalloc(code, llr, syn, F, max_iter, params, keys, conv, iters)
        torch.cuda.synchronize()
        assert torch.equal(keys, ref.keys), f"call {call}: key bits differ"
        assert torch.equal(conv, ref.converged), f"call {call}: flags differ"
        assert torch.equal(iters, ref.iters), f"call {call}: iteration counts differ"
        assert int(iters.min()) >= 1


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    code = q.create_code_from(synth.rate002_code(20000))  # ~13.7 MB per frame
    llr = torch.zeros(2 * code.n, dtype=torch.float32, device="cuda")
    syn = torch.zeros(2 * ((code.m + 31) // 32), dtype=torch.int32, device="cuda")
    keys, conv, iters = _outputs(code, 2)
    with pytest.raises(q.QcldpcError, match="UNSUPPORTED"):
        q.qcldpc_decode_noalloc(code, llr, syn, 2, 5, None, keys, conv, iters)
