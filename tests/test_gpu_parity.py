"""GPU-vs-oracle parity through the C ABI (libqcldpc).

Bars (bit-exact for integer work, a stated tolerance for floating point):
* syndromes, key bits, convergence flags, iteration counts: identical;
* 8-D maps: |gpu - ref| <= 16 u |M_b| |X_b| scale per block of eight
  (u = 2^-24; an 8-term FP32 dot product per output, see llr_tolerance);
* posteriors after a fixed iteration count: |L_gpu - L_ref| <=
  1e-3 max(|L_ref|, 0.1) for every variable node.
"""
import numpy as np
import pytest

import oracle
import synth
from frames import make_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1702_07740_gb300 import qcldpc as q  # noqa: E402

U32 = 2.0 ** -24
POST_RTOL = 1e-3
POST_FLOOR = 0.1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device visible")
    q.load()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.view(dtype)
    return t.cuda()


def packed(bits2d):
    return synth.pack_bits(bits2d).astype(np.uint32)


def gpu_syndrome(code, bits2d):
    F = bits2d.shape[0]
    wm = (code.m + 31) // 32
    syn = torch.zeros(F * wm, dtype=torch.int32, device="cuda")
    q.qcldpc_syndrome(code, dev(packed(bits2d).view(np.int32).reshape(-1)), syn, F)
    torch.cuda.synchronize()
    return synth.unpack_bits(syn.cpu().numpy().view(np.uint32).reshape(F, wm), code.m)


def gpu_llr(fr):
    n = fr.x32.size
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(dev(fr.x32.reshape(-1)), dev(fr.m32.reshape(-1)), n, fr.snr, out)
    torch.cuda.synchronize()
    return out


def llr_tolerance(x32, m32, snr):
    """Per element: an FP32 octonion product output is an 8-term signed sum of
    products M_a X_b; its rounding error is below 8 u sum |M_a X_b| <=
    8 u |M_b| |X_b| (Cauchy-Schwarz), doubled for the final scaling and slack."""
    xb = np.linalg.norm(x32.reshape(-1, 8).astype(np.float64), axis=1)
    mb = np.linalg.norm(m32.reshape(-1, 8).astype(np.float64), axis=1)
    return np.repeat(16 * U32 * xb * mb * snr / 4.0, 8) + 1e-30


def decode_soft(code, llr, syn2d, F, max_iter, et_start=None, **pk):
    params = q.qcldpc_params_init(soft_output=1, **pk)
    if et_start is not None:
        params.et_start = et_start
    dec = q.Decoder(code, F, params, soft=True)
    wm = (code.m + 31) // 32
    syn = dev(packed(syn2d).view(np.int32).reshape(-1))
    assert syn.numel() == F * wm
    dec.decode(llr, syn, max_iter)
    torch.cuda.synchronize()
    wk = (code.k + 31) // 32
    keys = synth.unpack_bits(dec.keys.cpu().numpy().view(np.uint32).reshape(F, wk), code.k)
    post = dec.posterior.cpu().numpy().reshape(F, code.n).astype(np.float64)
    return keys, dec.converged.cpu().numpy(), dec.iters.cpu().numpy(), post


def assert_posteriors_close(post, ref, what=""):
    err = np.abs(post - ref) / np.maximum(np.abs(ref), POST_FLOOR)
    assert err.max() <= POST_RTOL, (
        f"{what}: max scaled error {err.max():.3e} (p99.9 {np.quantile(err, 0.999):.3e})")
    return err


# ------------------------------------------------------------------ codes

def odd_code(Z):
    """Small irregular code: ragged Z, non-zero diagonal shifts, one row with
    two degree-1 nodes, one row with none, an empty column, and key bits that
    include a degree-1 column (k = 3Z covers columns 0, 1, 2)."""
    rng = np.random.default_rng(Z)
    mb, nb = 5, 8
    ents = set()
    for r in range(mb):
        for c in range(2):
            k = min(1 + int(rng.integers(0, 2)), Z)
            for s in rng.choice(Z, size=k, replace=False):
                ents.add((r, c, int(s)))
    for r in range(4):                      # columns 2..5: degree-1 on rows 0..3
        ents.add((r, 2 + r, int(rng.integers(Z))))
    ents.add((1, 7, int(rng.integers(Z))))  # column 7: second degree-1 node of row 1
    rows, cols, shifts = zip(*sorted(ents))  # column 6 stays empty; row 4 has no diagonal
    return {"mb": mb, "nb": nb, "Z": Z, "row": np.array(rows), "col": np.array(cols),
            "shift": np.array(shifts)}


# ---------------------------------------------------------------- syndrome

@pytest.mark.parametrize("maker, Z, F", [
    (synth.rate002_code, 512, 3), (odd_code, 37, 4), (odd_code, 5, 2), (odd_code, 1, 2),
    (synth.rate005_code, 100, 2), (synth.rate010_code, 96, 2),
])
def test_syndrome_bit_exact(maker, Z, F):
    d = maker(Z)
    code = oracle.Code.from_dict(d)
    rng = np.random.default_rng(Z * 7 + F)
    bits = rng.integers(0, 2, (F, code.n)).astype(np.uint8)
    gcode = q.create_code_from(d)
    got = gpu_syndrome(gcode, bits)
    ref = np.stack([oracle.syndrome(code, b) for b in bits])
    np.testing.assert_array_equal(got, ref)


def test_syndrome_full_size_bit_exact():
    d = synth.rate002_code(20000)
    code = oracle.Code.from_dict(d)
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2, (16, code.n)).astype(np.uint8)
    got = gpu_syndrome(q.create_code_from(d), bits)
    for f in (0, 7, 15):
        np.testing.assert_array_equal(got[f], oracle.syndrome(code, bits[f]))


# ------------------------------------------------------------------ 8-D map

@pytest.mark.parametrize("Z, F, snr", [(512, 2, 0.029), (20000, 1, 0.029), (40, 1, 0.5)])
def test_bob_message_and_llr_8d(Z, F, snr):
    fr = make_frames(synth.rate002_code(Z), snr, F)
    n = fr.x32.size
    m_gpu = torch.empty(n, dtype=torch.float32, device="cuda")
    q.qcldpc_bob_message_8d(dev(fr.y32.reshape(-1)),
                            dev(packed(fr.bits.reshape(1, -1)).view(np.int32).reshape(-1)),
                            n, m_gpu)
    torch.cuda.synchronize()
    m_ref = np.concatenate([oracle.bob_message(fr.y32[f].astype(np.float64), fr.bits[f])
                            for f in range(F)])
    ub = np.repeat(np.linalg.norm(fr.y32.reshape(-1, 8).astype(np.float64), axis=1), 8)
    assert np.all(np.abs(m_gpu.cpu().numpy() - m_ref) <= 16 * U32 * np.sqrt(8) * ub + 1e-30)

    got = gpu_llr(fr).cpu().numpy().astype(np.float64)
    ref = fr.q64.reshape(-1)
    tol = llr_tolerance(fr.x32, fr.m32, snr) + 2 * U32 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("d", [1, 2, 4, 8])
def test_bob_message_and_llr_all_dimensions(d):
    """The d-dimensional maps of Sec. II-C against the oracle (Z=64, 2 frames)."""
    fr = make_frames(synth.rate002_code(64), 0.1, 2, d=d)
    n = fr.x32.size
    m_gpu = torch.empty(n, dtype=torch.float32, device="cuda")
    q.qcldpc_bob_message(d, dev(fr.y32.reshape(-1)),
                         dev(packed(fr.bits.reshape(1, -1)).view(np.int32).reshape(-1)), n, m_gpu)
    llr = torch.empty(n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr(d, dev(fr.x32.reshape(-1)), dev(fr.m32.reshape(-1)), n, fr.snr, llr)
    torch.cuda.synchronize()
    m_ref = np.concatenate([oracle.bob_message(fr.y32[f].astype(np.float64), fr.bits[f], d=d)
                            for f in range(fr.F)])
    yb = np.repeat(np.linalg.norm(fr.y32.reshape(-1, d).astype(np.float64), axis=1), d)
    assert np.all(np.abs(m_gpu.cpu().numpy() - m_ref) <= 16 * U32 * np.sqrt(d) * yb + 1e-30)
    ref = fr.q64.reshape(-1)
    xb = np.linalg.norm(fr.x32.reshape(-1, d).astype(np.float64), axis=1)
    mb = np.linalg.norm(fr.m32.reshape(-1, d).astype(np.float64), axis=1)
    tol = np.repeat(16 * U32 * xb * mb * 2 * fr.snr / d, d) + 2 * U32 * np.abs(ref) + 1e-30
    assert np.all(np.abs(llr.cpu().numpy().astype(np.float64) - ref) <= tol)


def test_llr_rejects_bad_length_and_alignment():
    x = torch.zeros(24, device="cuda")
    with pytest.raises(q.QcldpcError, match="INVAL"):
        q.qcldpc_llr_8d(x, x, 12, 0.1, x)
    with pytest.raises(q.QcldpcError, match="ALIGN"):
        q.qcldpc_llr_8d(x[1:17], x[:16], 16, 0.1, x[:16])


# ----------------------------------------------------------------- decoding

@pytest.mark.parametrize("vn_pass", [0, 1])
@pytest.mark.parametrize("F", [1, 4])
def test_decode_fixed_iterations_matches_oracle(F, vn_pass):
    """Z=512 (n=25,600), SNR 0.029, 50 flooding iterations, no early stop;
    posteriors accumulated by the check pass (vn_pass 0) or summed by a
    separate variable pass (vn_pass 1)."""
    fr = make_frames(synth.rate002_code(512), 0.029, F)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    iters = 50
    keys, conv, its, post = decode_soft(code, llr, fr.syn, F, iters, et_start=iters + 1,
                                        vn_pass=vn_pass)
    for f in range(F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], iters,
                                          et_start=iters + 1)
        err = assert_posteriors_close(post[f], ref, f"frame {f}")
        assert its[f] == it == iters and conv[f] == int(cv)
        # decisions agree wherever the posterior is not within rounding of 0
        sure = np.abs(ref) > 1e-3
        np.testing.assert_array_equal((post[f] < 0)[sure], chat.astype(bool)[sure])
        print(f"frame {f}: max scaled err {err.max():.2e} p99.9 {np.quantile(err, 0.999):.2e}")


def test_decode_early_stop_matches_oracle():
    """Frames that converge at different iterations: identical stop iteration,
    flag and key bits; posteriors at the stop within tolerance."""
    fr = make_frames(synth.rate002_code(64), 0.08, 12)
    code = q.create_code_from(fr.code_dict)
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, fr.F, 60)
    n_conv = 0
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 60)
        assert (its[f], conv[f]) == (it, int(cv)), f"frame {f}"
        if cv:
            # key bits must be identical on every frame both sides converge on;
            # a frame that never converges oscillates, and after 60 iterations
            # FP32 and FP64 trajectories may part, so only its flag is compared
            n_conv += 1
            np.testing.assert_array_equal(keys[f], chat[: fr.code.k], f"frame {f}")
            assert_posteriors_close(post[f], ref, f"frame {f}")
    assert 0 < n_conv < fr.F


def test_decode_et_start_delays_the_stop_test():
    fr = make_frames(synth.rate002_code(64), 0.12, 4)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    for et in (1, 9):
        _, conv, its, _ = decode_soft(code, llr, fr.syn, fr.F, 40, et_start=et)
        for f in range(fr.F):
            _, _, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 40, et_start=et)
            assert (its[f], conv[f]) == (it, int(cv))
            if cv:
                assert its[f] >= et


def test_decode_zero_iterations_returns_channel_decisions():
    fr = make_frames(synth.rate002_code(64), 0.05, 2)
    code = q.create_code_from(fr.code_dict)
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, fr.F, 0)
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 0)
        assert its[f] == 0 and conv[f] == int(cv)
        np.testing.assert_array_equal(keys[f], chat[: fr.code.k])
        assert_posteriors_close(post[f], ref)


@pytest.mark.parametrize("clip", [2.0, 5.0])
def test_binding_clip_matches_oracle(clip):
    """A clip low enough to bind on check outputs (psi(clip) above the floor
    of the psi sums): the GPU folds the output clip into that floor, the
    oracle clips each message; posteriors agree to the usual tolerance."""
    fr = make_frames(synth.rate002_code(512), 0.3, 2)
    code = q.create_code_from(fr.code_dict)
    iters = 20
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, fr.F, iters, et_start=iters + 1,
                                        clip=clip)
    for f in range(fr.F):
        ref, _, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], iters, et_start=iters + 1,
                                       clip=clip)
        assert_posteriors_close(post[f], ref, f"clip {clip} frame {f}")
        assert its[f] == it and conv[f] == int(cv)


@pytest.mark.parametrize("Z", [700, 1500, 2000, 2052])
def test_check_block_widths_match_oracle(Z):
    """The check pass sizes its blocks to Z: 1024-check tiles when those fill
    the row (Z = 2000: two tiles, the second 976 checks), else the fewest
    warps that cover the row in as many tiles (Z = 700: one 768-check tile of
    192 threads; Z = 1500: two, the second 732 checks; Z = 2052: three, the
    last 516 checks). Soft output and the stop test on both kernel forms."""
    fr = make_frames(synth.rate002_code(Z), 0.12, 2)
    code = q.create_code_from(fr.code_dict)
    iters = 12
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, fr.F, iters, et_start=6)
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], iters, et_start=6)
        assert (its[f], conv[f]) == (it, int(cv)), f"Z={Z} frame {f}"
        assert_posteriors_close(post[f], ref, f"Z={Z} frame {f}")


@pytest.mark.parametrize("Z", [1, 2, 5, 37, 100])
def test_decode_ragged_and_irregular_codes(Z):
    d = odd_code(Z)
    fr = make_frames(d, 0.3, 3)
    code = q.create_code_from(d)
    llr = gpu_llr(fr)
    iters = 15
    keys, conv, its, post = decode_soft(code, llr, fr.syn, fr.F, iters, et_start=iters + 1)
    for f in range(fr.F):
        ref, chat, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], iters,
                                          et_start=iters + 1)
        assert_posteriors_close(post[f], ref, f"Z={Z} frame {f}")
        assert conv[f] == int(cv)
        sure = np.abs(ref[: fr.code.k]) > 1e-3
        np.testing.assert_array_equal(keys[f][sure], chat[: fr.code.k][sure])


def test_decode_is_deterministic():
    fr = make_frames(synth.rate002_code(512), 0.029, 2)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    outs = [decode_soft(code, llr, fr.syn, fr.F, 20, et_start=99) for _ in range(3)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o[3], outs[0][3])
        np.testing.assert_array_equal(o[0], outs[0][0])


def test_stream_launch_mode_matches_graph_mode():
    """launch_mode 1 (host-enqueued passes) computes exactly what the graph does."""
    fr = make_frames(synth.rate002_code(64), 0.08, 6)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    a = decode_soft(code, llr, fr.syn, fr.F, 40)
    b = decode_soft(code, llr, fr.syn, fr.F, 40, launch_mode=1)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_decode_zero_frames_and_bad_args():
    code = q.create_code_from(synth.rate002_code(64))
    dec = q.Decoder(code, 1)
    x = torch.zeros(code.n, device="cuda")
    s = torch.zeros((code.m + 31) // 32, dtype=torch.int32, device="cuda")
    q.qcldpc_decode(code, x, s, 0, 10, None, dec.keys, dec.converged, dec.iters,
                    dec.workspace, dec.ws_bytes)
    with pytest.raises(q.QcldpcError, match="NOMEM"):
        q.qcldpc_decode(code, x, s, 1, 10, None, dec.keys, dec.converged, dec.iters,
                        dec.workspace, 64)
    with pytest.raises(q.QcldpcError, match="INVAL"):
        q.qcldpc_decode(code, x, s, 1, -1, None, dec.keys, dec.converged, dec.iters,
                        dec.workspace, dec.ws_bytes)


# ------------------------------------------------- full size (n = 10^6)

def _oracle_decodes(jobs):
    """oracle.decode on several frames at once, one host thread each (the C
    oracle runs without the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        futs = [ex.submit(oracle.decode, *a, **k) for a, k in jobs]
        return [f.result() for f in futs]


def test_full_size_batch_parity_50_iterations():
    """Z=20,000 (n=10^6), 16 frames in one launch as timed by the benchmark;
    frames 0 and 15 compared with the oracle after 50 iterations."""
    F, iters = 16, 50
    d = synth.rate002_code(20000)
    fr_edges = make_frames(d, 0.029, 1)  # frame 0
    fr_last = make_frames(d, 0.029, 1, seed0=synth.frame_seed(F - 1))
    code = q.create_code_from(d)
    n = fr_edges.code.n
    # middle frames: any seeded data (not compared)
    x = np.concatenate([fr_edges.x32] + [fr_edges.x32 * 0.5] * (F - 2) + [fr_last.x32])
    m = np.concatenate([fr_edges.m32] + [fr_edges.m32] * (F - 2) + [fr_last.m32])
    syn = np.concatenate([fr_edges.syn] + [fr_edges.syn] * (F - 2) + [fr_last.syn])
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(dev(x.reshape(-1)), dev(m.reshape(-1)), F * n, 0.029, llr)
    keys, conv, its, post = decode_soft(code, llr, syn, F, iters, et_start=iters + 1)
    pairs = ((0, fr_edges), (F - 1, fr_last))
    refs = _oracle_decodes([((fr.code, fr.q64[0], fr.syn[0], iters), dict(et_start=iters + 1))
                            for _, fr in pairs])
    for (f, fr), (ref, chat, it, cv) in zip(pairs, refs):
        err = assert_posteriors_close(post[f], ref, f"frame {f}")
        assert its[f] == it == iters and conv[f] == int(cv)
        print(f"n=10^6 frame {f}, {iters} iterations: max scaled err {err.max():.2e}")


def test_results_do_not_depend_on_the_batch():
    """A frame decodes to the same bits alone and in a batch, although the
    launch shapes differ (variable pass: 1 node per thread alone, 3 in a
    16-frame batch): a check's arithmetic does not depend on its tile, and
    the variable pass adds each node's partial sums in a fixed order.
    n = 10^6: one frame alone against the same frame first and last in a
    16-frame batch."""
    F, iters = 16, 6
    d = synth.rate002_code(20000)
    fr = make_frames(d, 0.029, 1)
    code = q.create_code_from(d)
    n = fr.code.n
    x = np.concatenate([fr.x32] + [fr.x32 * 0.5] * (F - 2) + [fr.x32])
    m = np.concatenate([fr.m32] * F)
    syn = np.concatenate([fr.syn] * F)
    llr = torch.empty(F * n, dtype=torch.float32, device="cuda")
    q.qcldpc_llr_8d(dev(x.reshape(-1)), dev(m.reshape(-1)), F * n, 0.029, llr)
    batch = decode_soft(code, llr, syn, F, iters, et_start=iters + 1)
    alone = decode_soft(code, llr[:n].clone(), fr.syn, 1, iters, et_start=iters + 1)
    for f in (0, F - 1):
        np.testing.assert_array_equal(batch[3][f], alone[3][0], f"frame {f} posteriors")
        np.testing.assert_array_equal(batch[0][f], alone[0][0], f"frame {f} keys")
        assert (batch[1][f], batch[2][f]) == (alone[1][0], alone[2][0])


def test_full_size_converged_frames_match_the_oracle():
    """At SNR 0.15 n=10^6 frames converge within a few iterations: the hard
    decisions of every converged frame satisfy H C = s (checked by the
    oracle's syndrome), the key bits are those decisions, and on every frame
    both decoders converge on, the key bits, stop iteration and flag equal
    the oracle's."""
    F = 4
    fr = make_frames(synth.rate002_code(20000), 0.15, F)
    code = q.create_code_from(fr.code_dict)
    keys, conv, its, post = decode_soft(code, gpu_llr(fr), fr.syn, F, 60)
    refs = _oracle_decodes([((fr.code, fr.q64[f], fr.syn[f], 60), {}) for f in range(F)])
    both = 0
    for f in range(F):
        chat = (post[f] < 0).astype(np.uint8)
        ok = (oracle.syndrome(fr.code, chat) == fr.syn[f]).all()
        assert ok == bool(conv[f])
        np.testing.assert_array_equal(keys[f], chat[: fr.code.k])
        _, chat_ref, it_ref, cv_ref = refs[f]
        if conv[f] and cv_ref:
            both += 1
            np.testing.assert_array_equal(keys[f], chat_ref[: fr.code.k], f"frame {f}")
            assert its[f] == it_ref, f"frame {f}"
    print("n=10^6, SNR 0.15: GPU flags", conv.tolist(), "oracle flags", [int(r[3]) for r in refs])
    assert both >= 1


def test_launch_shapes_give_identical_bits_and_autotune_picks_the_fastest():
    """Every check-block width and variable-pass shape decodes to the same
    bits (posteriors included); qcldpc_autotune_shapes times them on the
    state of the last decode and returns the fastest."""
    fr = make_frames(synth.rate002_code(2000), 0.12, 4)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    iters = 10
    ref = decode_soft(code, llr, fr.syn, fr.F, iters, et_start=5)
    shapes = [dict(cn_threads=c) for c in q.SHAPE_CN_THREADS] + \
             [dict(vn_nodes=v, vn_split=s) for v, s in q.SHAPE_VN]
    for sh in shapes:
        got = decode_soft(code, llr, fr.syn, fr.F, iters, et_start=5, **sh)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b, str(sh))
    params = q.qcldpc_params_init(soft_output=1)
    dec = q.Decoder(code, fr.F, params, soft=True)
    syn = dev(packed(fr.syn).view(np.int32).reshape(-1))
    dec.decode(llr, syn, iters)
    best, tc, tv = q.qcldpc_autotune_shapes(code, fr.F, dec.workspace, dec.ws_bytes, params, reps=3)
    assert set(tc) == set(q.SHAPE_CN_THREADS) and set(tv) == set(q.SHAPE_VN)
    assert all(t > 0 for t in list(tc.values()) + list(tv.values()))
    assert best.cn_threads == min(tc, key=tc.get)
    assert (best.vn_nodes, best.vn_split) == min(tv, key=tv.get)
    assert best.soft_output == 1  # the other options are the caller's
    print("shape ms:", {k: round(v, 4) for k, v in tc.items()}, {k: round(v, 4) for k, v in tv.items()})
    for bad in (dict(cn_threads=48), dict(cn_threads=512), dict(vn_nodes=4), dict(vn_split=3)):
        with pytest.raises(q.QcldpcError, match="INVAL"):
            decode_soft(code, llr, fr.syn, fr.F, iters, **bad)


def test_a_staged_wait_that_runs_out_fails_the_decode_without_a_fault(monkeypatch):
    """Failure detection on the device, without a fault: under the library's
    test switch every check-pass block expects 16 bytes more than its bulk
    copies deliver, so its bounded mbarrier wait runs out. The blocks set the
    device error word and return; the decode stops every frame with
    converged = -1, and the context stays usable: the next decode matches
    the oracle."""
    fr = make_frames(synth.rate002_code(512), 0.05, 2)
    code = q.create_code_from(fr.code_dict)
    llr = gpu_llr(fr)
    monkeypatch.setenv("QCLDPC_TEST_STALL", "1")
    keys, conv, its, post = decode_soft(code, llr, fr.syn, fr.F, 10)
    assert (conv == -1).all() and (its == 0).all()
    monkeypatch.delenv("QCLDPC_TEST_STALL")
    keys, conv, its, post = decode_soft(code, llr, fr.syn, fr.F, 10, et_start=11)
    for f in range(fr.F):
        ref, _, it, cv = oracle.decode(fr.code, fr.q64[f], fr.syn[f], 10, et_start=11)
        assert its[f] == it and conv[f] == int(cv)
        assert_posteriors_close(post[f], ref, f"frame {f} after the failed decode")
