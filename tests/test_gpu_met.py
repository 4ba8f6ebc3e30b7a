"""The decoder on codes sampled from the paper's multi-edge distribution
(1568 x 1600 base matrices: tables in the device table arena, type-1 rows of
degree 7 on the generic check-node path) against the FP64 oracle. Bars as in
test_gpu_parity."""
import numpy as np
import pytest

import oracle
import synth
from frames import make_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1702_07740_gb300 import qcldpc as q  # noqa: E402
from test_gpu_parity import assert_posteriors_close, decode_soft, gpu_llr  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    q.load()


@pytest.mark.parametrize("Z, F", [(3, 2), (16, 3)])
def test_met_code_fixed_iterations_match_oracle(Z, F):
    fr = make_frames(synth.met_code(Z), 0.05, F)
    code = q.create_code_from(fr.code_dict)
    iters = 25
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, F, iters, et_start=iters + 1)
    for f in range(F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], iters, et_start=iters + 1)
        err = assert_posteriors_close(post[f], ref, f"Z={Z} frame {f}")
        assert its[f] == it and conv[f] == int(cv)
        print(f"MET Z={Z} frame {f}: max scaled err {err.max():.2e}")


def test_met_code_early_stop_matches_oracle():
    fr = make_frames(synth.met_code(16), 0.2, 4)
    code = q.create_code_from(fr.code_dict)
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, fr.F, 100)
    n_conv = 0
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 100)
        assert (its[f], conv[f]) == (it, int(cv)), f"frame {f}"
        if cv:
            n_conv += 1
            np.testing.assert_array_equal(keys[f], chat[: fr.code.k])
    assert n_conv > 0


def test_met_code_full_size_few_iterations():
    """n = 10^6 (Z = 625), 4 frames; frame 0 against the oracle after 3 iterations."""
    d = synth.met_code(625)
    fr = make_frames(d, 0.03, 1)
    code = q.create_code_from(d)
    F = 4
    x = np.concatenate([fr.x32] * F)
    m = np.concatenate([fr.m32] * F)
    syn = np.concatenate([fr.syn] * F)
    n = fr.code.n
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(torch.from_numpy(x.reshape(-1)).cuda(), torch.from_numpy(m.reshape(-1)).cuda(),
                    F * n, 0.03, llr)
    _, _, _, post = decode_soft(code, llr, syn, F, 3, et_start=4)
    ref, _, _, _ = oracle.decode(fr.code, fr.q64[0], fr.syn[0], 3, et_start=4)
    for f in range(F):
        assert_posteriors_close(post[f], ref, f"frame {f}")


def test_table_arena_fills_with_nomem_and_frees_on_destroy():
    """Code tables share a 64 MiB device arena: codes take their block on the
    first launching call and give it back when destroyed."""
    d = synth.met_code(2)
    bits = torch.zeros(1600 * 2 // 32, dtype=torch.int32, device="cuda")
    syn = torch.zeros((1568 * 2 + 31) // 32, dtype=torch.int32, device="cuda")
    codes, failed = [], None
    for i in range(400):  # ~0.4 MB each: the 64 MiB arena holds about 160
        c = q.create_code_from(d)
        try:
            q.qcldpc_syndrome(c, bits, syn, 1)
        except q.QcldpcError as e:
            failed = e
            break
        codes.append(c)
    assert failed is not None and "NOMEM" in str(failed)
    assert 20 <= len(codes) < 400  # other live codes of the session hold blocks too
    # give back two blocks: the next code fits again
    del codes[:2]
    import gc
    gc.collect()
    c = q.create_code_from(d)
    q.qcldpc_syndrome(c, bits, syn, 1)
    torch.cuda.synchronize()
    del codes, c
    gc.collect()


@pytest.mark.parametrize("schedule", [0, 1])
def test_met_code_in_a_pool_decodes_as_alone(schedule):
    """The 1568 x 1600 multi-edge code (column lists staged in shared memory
    by the variable pass, variable-width check blocks) in a 3-slot pool with
    frames loaded at different times: key bits, flag and stop iteration as
    decoded alone, flooding and layered (8 row groups)."""
    d = synth.met_code(16)
    code = q.create_code_from(d)
    fr = make_frames(d, 0.2, 3)
    llr = gpu_llr(fr)
    n = fr.code.n
    syn = torch.from_numpy(synth.pack_bits(fr.syn).view(np.int32)).cuda()
    params = q.qcldpc_params_init(schedule=schedule, layers=8 if schedule else 0)
    max_iter = 80
    alone = []
    for f in range(fr.F):
        dec = q.Decoder(code, 1, params)
        dec.decode(llr[f * n:(f + 1) * n], syn[f], max_iter)
        torch.cuda.synchronize()
        alone.append((dec.keys.cpu(), int(dec.converged[0]), int(dec.iters[0])))
    pool = q.Pool(code, 3, max_iter, params)
    ids = torch.arange(3, dtype=torch.int32, device="cuda")
    for f in range(fr.F):
        q.qcldpc_pool_load(pool, 1, ids[f:f + 1], llr[f * n:(f + 1) * n], syn[f])
        q.qcldpc_pool_step(pool, 4)
    for _ in range(max_iter + 2):
        if all(int(s) == 2 for s in pool.state.cpu()):
            break
        q.qcldpc_pool_step(pool, 1)
    wk = (code.k + 31) // 32
    keys = torch.empty(fr.F * wk, dtype=torch.int32, device="cuda")
    conv = torch.empty(fr.F, dtype=torch.int32, device="cuda")
    its = torch.empty(fr.F, dtype=torch.int32, device="cuda")
    q.qcldpc_pool_collect(pool, fr.F, ids, keys, conv, its)
    torch.cuda.synchronize()
    for f in range(fr.F):
        ak, ac, ai = alone[f]
        assert (int(conv[f]), int(its[f])) == (ac, ai), f"frame {f}"
        assert torch.equal(keys[f * wk:(f + 1) * wk].cpu(), ak.view(-1)), f"frame {f}"
    assert sum(a[1] for a in alone) >= 1
