"""Studies beside bench.py's throughput line (``bench.py --study ...``).

* ``fer``: the same seeded n = 10^6 frames (rates 0.02, 0.05, 0.10) decoded
  with edge messages stored in FP32, FP16 and int8 (arithmetic FP32); per
  format and operating point the frame error rate
  with its Wilson 95 % interval, the paired difference to FP32 with its 95 %
  interval, mean iterations and decoded Mbit/s.
* ``batch``: 256 frames drawn uniformly from nine codes (rates 0.02, 0.05
  and 0.10, each at n = 10^5, 4*10^5 and 10^6) decoded together in one
  batched decode (one graph launch, each code in its own device-side loop),
  and by frame pools stepped in one graph launch per step (FP16 and FP32
  messages), against the plain FP32 decoder run one frame at a time and one
  code at a time. Each variant decodes the mix --mix-reps times in a row.
* ``schedule``: the library's autotuner (flooding vs layered with 2, 7 and
  mb row groups) on a 16-frame sample of each FER operating point.
* ``et``: delayed early termination, an SNR -> et_start table built from
  sample frames, against the stop test from iteration 1.
* ``serve``: Poisson arrivals of frames of the same mix into the
  continuous-batching server (FP16 messages) at offered loads from 10 % to
  120 % of its measured capacity; p50/p99 frame latency and served Mbit/s,
  next to a first-in-first-out server that decodes one frame at a time with
  the plain FP32 decoder on the same arrivals.

Frames are seeded synthetic channel draws made on the device with torch's
Philox generator (x ~ N(0,1), y = x + N(0, 1/SNR), uniform bits); Bob's
message, the syndrome and Alice's LLRs then come from the library's own
kernels. Every variant of a study decodes the same frames, so differences in
frame errors are paired. A frame error is a key that differs from Bob's first
k bits (converged or not).
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

import synth
from bench import wilson
from paper_1702_07740_gb300 import qcldpc as q
from paper_1702_07740_gb300 import serve

# The mixed-rate workload: three rates, each at n = 10^5, 4*10^5 and 10^6.
RATES = (("r002", synth.rate002_code, (2000, 8000, 20000)),
         ("r005", synth.rate005_code, (5000, 20000, 50000)),
         ("r010", synth.rate010_code, (10000, 40000, 100000)))
MIX = tuple((f"{name}_z{Z}", mk, Z, ri) for ri, (name, mk, Zs) in enumerate(RATES) for Z in Zs)
FMT = {"fp32": 0, "fp16": 1, "int8": 2}


# ------------------------------------------------------------------ frames

def pack_dev(bits: torch.Tensor) -> torch.Tensor:
    """0/1 int32 [F, n] (n a multiple of 32) -> int32 [F, n/32], LSB first."""
    F, n = bits.shape
    sh = torch.arange(32, device=bits.device, dtype=torch.int64)
    w = (bits.view(F, n // 32, 32).to(torch.int64) << sh).sum(-1)
    w = torch.where(w >= 2 ** 31, w - 2 ** 32, w)
    return w.to(torch.int32)


def make_frames(code, F: int, snr: float, seed: int):
    """(llr float[F n], syndrome int32[F ceil(m/32)], Bob's key int32[F, ceil(k/32)])."""
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    n, k, m = code.n, code.k, code.m
    wm, wk = (m + 31) // 32, (k + 31) // 32
    x = torch.randn(F * n, generator=g, device=dev)
    y = x + torch.randn(F * n, generator=g, device=dev) * (1.0 / snr) ** 0.5
    words = pack_dev(torch.randint(0, 2, (F, n), generator=g, device=dev, dtype=torch.int32))
    msg = torch.empty_like(x)
    q.qcldpc_bob_message_8d(y, words.view(-1), F * n, msg)
    del y
    syn = torch.empty(F * wm, dtype=torch.int32, device=dev)
    q.qcldpc_syndrome(code, words.view(-1), syn, F)
    llr = torch.empty_like(x)
    q.qcldpc_llr_8d(x, msg, F * n, snr, llr)
    key = words[:, :wk].clone()
    if k % 32:
        key[:, -1] &= (1 << (k % 32)) - 1
    return llr, syn, key


def paired(e_ref: np.ndarray, e: np.ndarray) -> dict:
    """Paired FER difference (e - e_ref) with a 95 % normal interval."""
    N = len(e)
    b = int(((e_ref == 0) & (e == 1)).sum())
    c = int(((e_ref == 1) & (e == 0)).sum())
    d = (b - c) / N
    se = math.sqrt(max(b + c - (b - c) ** 2 / N, 0.0)) / N
    return {"only_this_fails": b, "only_ref_fails": c, "diff": d,
            "diff_ci95": [d - 1.96 * se, d + 1.96 * se]}


def fer_entry(err: np.ndarray) -> dict:
    k, n = int(err.sum()), len(err)
    return {"frames": n, "errors": k, "fer": k / n, "fer_wilson95": list(wilson(k, n))}


def parse_floats(s: str):
    return [float(x) for x in s.split(",") if x]


def emit(line: dict):
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- fer

# n = 10^6 member of each rate, for the FER study
FER_CODES = {"met": (synth.met_code, 625, "rate 0.02 multi-edge (paper's distribution)"),
             "met6": (lambda Z: synth.met_code(Z, girth6=True), 625,
                      "rate 0.02 multi-edge (paper's distribution), shifts without 4-cycles"),
             "r002": (synth.rate002_code, 20000, "rate 0.02"),
             "r005": (synth.rate005_code, 50000, "rate 0.05"),
             "r010": (synth.rate010_code, 100000, "rate 0.10")}


def study_fer(args):
    F = 50
    nb = (args.study_frames + F - 1) // F
    for si, item in enumerate(args.fer_points.split(",")):
        cname, snr = item.split(":")
        snr = float(snr)
        mk, Z, label = FER_CODES[cname]
        code = q.create_code_from(mk(Z))
        wk = (code.k + 31) // 32
        fmts = {f: FMT[f] for f in args.fer_formats.split(",")}
        decs = {f: q.Decoder(code, F, q.qcldpc_params_init(msg_format=fmts[f])) for f in fmts}
        acc = {f: {"err": [], "conv": [], "iters": [], "sec": 0.0} for f in fmts}
        for b in range(nb):
            llr, syn, key = make_frames(code, F, snr, seed=7_000_000 + 10_000 * si + b)
            for f, dec in decs.items():
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                dec.decode(llr, syn, args.max_iter)
                e1.record()
                e1.synchronize()
                acc[f]["sec"] += e0.elapsed_time(e1) / 1e3
                acc[f]["err"].append((dec.keys.view(F, wk) != key).any(1).cpu().numpy())
                acc[f]["conv"].append(dec.converged.cpu().numpy())
                acc[f]["iters"].append(dec.iters.cpu().numpy())
            del llr, syn, key
        ref = np.concatenate(acc[next(iter(fmts))]["err"]).astype(np.int64)
        out = {"study": "fer", "code": f"{label}, Z={Z}, n={code.n}", "snr": snr,
               "max_iter": args.max_iter, "frames_per_decode": F, "formats": {}}
        for f in fmts:
            e = np.concatenate(acc[f]["err"]).astype(np.int64)
            conv = np.concatenate(acc[f]["conv"])
            its = np.concatenate(acc[f]["iters"])
            ent = fer_entry(e)
            ent.update({"converged": int((conv == 1).sum()),
                        "undetected": int(((conv == 1) & (e == 1)).sum()),
                        "mean_iters": float(its.mean()),
                        "mbps": len(e) * code.n / acc[f]["sec"] / 1e6})
            if f != "fp32" and "fp32" in fmts:
                ent["vs_fp32"] = paired(ref, e)
            out["formats"][f] = ent
        emit(out)


# ------------------------------------------------------------------- batch

def mix_setup(args, frames_per_code):
    """Codes of the mix and their frames; the SNR is set per rate."""
    snr_of_rate = parse_floats(args.mix_snrs)
    codes, inputs, snrs = {}, {}, {}
    for i, (name, mk, Z, ri) in enumerate(MIX):
        if frames_per_code.get(name, 0) == 0:
            continue
        codes[name] = q.create_code_from(mk(Z))
        snrs[name] = snr_of_rate[ri]
        inputs[name] = make_frames(codes[name], frames_per_code[name], snrs[name],
                                   seed=8_000_000 + 1000 * i)
    return codes, inputs, snrs


def split_mix(total: int, seed: int = 4) -> dict:
    """Frames per code of a seeded uniform draw over the codes of the mix."""
    draw = np.random.default_rng(seed).integers(0, len(MIX), total)
    return {name: int((draw == i).sum()) for i, (name, _, _, _) in enumerate(MIX)}


class PoolBatch:
    """One pool per code with a slot for every frame of the mix. ``run``
    loads all frames, steps the pools together (one graph launch per step)
    until every slot stopped, and collects; the slots are free again after."""

    def __init__(self, codes, counts, fmt, max_iter, passes=8):
        params = q.qcldpc_params_init(msg_format=FMT[fmt])
        self.codes, self.counts, self.passes = codes, counts, passes
        self.pools = {c: q.Pool(codes[c], counts[c], max_iter, params) for c in codes}
        self.ids = {c: torch.arange(counts[c], dtype=torch.int32, device="cuda") for c in codes}
        self.outs = {c: (torch.empty((counts[c], (codes[c].k + 31) // 32), dtype=torch.int32,
                                     device="cuda"),
                         torch.empty(counts[c], dtype=torch.int32, device="cuda"),
                         torch.empty(counts[c], dtype=torch.int32, device="cuda")) for c in codes}

    def run(self, inputs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in self.codes:
            llr, syn, _ = inputs[c]
            q.qcldpc_pool_load(self.pools[c], self.counts[c], self.ids[c], llr, syn)
        plist = list(self.pools.values())
        states = torch.cat([p.state for p in plist])
        while True:
            q.qcldpc_pools_step(plist, self.passes)
            torch.cat([p.state for p in plist], out=states)
            if bool((states == 2).all()):
                break
        for c in self.codes:
            q.qcldpc_pool_collect(self.pools[c], self.counts[c], self.ids[c], *self.outs[c])
        torch.cuda.synchronize()
        return time.perf_counter() - t0, self.outs


class PerFrame:
    """The plain FP32 decoder, one frame per call: each frame is copied into a
    fixed staging buffer, so every call reuses the decoder's cached graph
    (graphs are cached per argument set, buffer addresses included)."""

    def __init__(self, codes):
        self.codes = codes
        self.dec = {c: q.Decoder(codes[c], 1, q.qcldpc_params_init()) for c in codes}
        self.stage = {c: (torch.empty(codes[c].n, device="cuda"),
                          torch.empty((codes[c].m + 31) // 32, dtype=torch.int32, device="cuda"))
                      for c in codes}

    def decode(self, c, llr, syn, f, max_iter):
        n, wm = self.codes[c].n, (self.codes[c].m + 31) // 32
        self.stage[c][0].copy_(llr[f * n:(f + 1) * n])
        self.stage[c][1].copy_(syn[f * wm:(f + 1) * wm])
        d = self.dec[c]
        d.decode(self.stage[c][0], self.stage[c][1], max_iter)
        return d

    def run(self, inputs, counts, max_iter):
        res = {c: (torch.empty((counts[c], (self.codes[c].k + 31) // 32), dtype=torch.int32,
                               device="cuda"),
                   torch.empty(counts[c], dtype=torch.int32, device="cuda"),
                   torch.empty(counts[c], dtype=torch.int32, device="cuda")) for c in self.codes}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in self.codes:
            llr, syn, _ = inputs[c]
            for f in range(counts[c]):
                d = self.decode(c, llr, syn, f, max_iter)
                res[c][0][f].copy_(d.keys)
                res[c][1][f:f + 1].copy_(d.converged)
                res[c][2][f:f + 1].copy_(d.iters)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res


class MultiBatch:
    """Every frame of the mix in one batched decode (qcldpc_decode_multi):
    one graph launch runs all codes' passes side by side until every frame
    stopped."""

    def __init__(self, codes, counts, fmt):
        self.codes, self.counts = codes, counts
        self.names = list(codes)
        self.dec = q.MultiDecoder([codes[c] for c in self.names], [counts[c] for c in self.names],
                                  q.qcldpc_params_init(msg_format=FMT[fmt]))

    def run(self, inputs, max_iter):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.dec.decode([inputs[c][0] for c in self.names], [inputs[c][1] for c in self.names], max_iter)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res = {}
        for i, c in enumerate(self.names):
            wk, F = (self.codes[c].k + 31) // 32, self.counts[c]
            res[c] = (self.dec.keys[i][: F * wk].view(F, wk), self.dec.converged[i][:F], self.dec.iters[i][:F])
        return dt, res


class PerCode:
    """The plain FP32 decoder, one call per code with all of its frames."""

    def __init__(self, codes, counts):
        self.codes, self.counts = codes, counts
        self.dec = {c: q.Decoder(codes[c], counts[c], q.qcldpc_params_init()) for c in codes}

    def run(self, inputs, max_iter):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in self.codes:
            llr, syn, _ = inputs[c]
            self.dec[c].decode(llr, syn, max_iter)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res = {}
        for c in self.codes:
            d, wk = self.dec[c], (self.codes[c].k + 31) // 32
            res[c] = (d.keys.view(self.counts[c], wk), d.converged, d.iters)
        return dt, res


def summarise(codes, inputs, counts, sec, res):
    err_all, bits, info = [], 0, 0
    per = {}
    for c in codes:
        keys, conv, its = res[c]
        e = (keys != inputs[c][2]).any(1).cpu().numpy().astype(np.int64)
        cv = conv.cpu().numpy() == 1
        err_all.append(e)
        bits += counts[c] * codes[c].n
        info += int((e == 0).sum()) * codes[c].k
        # undetected: the decoder stopped on a codeword of the coset that is
        # not Bob's (H C = s holds, the key differs); detected: no convergence
        per[c] = {"frames": counts[c], "errors": int(e.sum()),
                  "undetected": int((cv & (e == 1)).sum()), "detected": int((~cv & (e == 1)).sum()),
                  "converged": int(cv.sum()),
                  "mean_iters": float(its.float().mean().item()),
                  "max_iters": int(its.max().item())}
    e = np.concatenate(err_all)
    out = fer_entry(e)
    out.update({"seconds": sec, "mbps": bits / sec / 1e6, "info_mbps": info / sec / 1e6,
                "frames_per_s": len(e) / sec, "per_code": per})
    return out, e


def study_batch(args):
    counts = {c: k for c, k in split_mix(args.mix_frames).items() if k > 0}
    codes, inputs, snrs = mix_setup(args, counts)
    pb16 = PoolBatch(codes, counts, "fp16", args.max_iter)
    pb32 = PoolBatch(codes, counts, "fp32", args.max_iter)
    mb16, mb32 = MultiBatch(codes, counts, "fp16"), MultiBatch(codes, counts, "fp32")
    per_frame, per_code = PerFrame(codes), PerCode(codes, counts)
    runs = {
        "multi_fp16": lambda: mb16.run(inputs, args.max_iter),
        "multi_fp32": lambda: mb32.run(inputs, args.max_iter),
        "pools_fp16": lambda: pb16.run(inputs),
        "pools_fp32": lambda: pb32.run(inputs),
        "per_frame_fp32": lambda: per_frame.run(inputs, counts, args.max_iter),
        "per_code_fp32": lambda: per_code.run(inputs, args.max_iter),
    }
    out = {"study": "batch", "frames": sum(counts.values()), "max_iter": args.max_iter,
           "mix": {name: {"Z": Z, "n": codes[name].n, "rate": codes[name].k / codes[name].n,
                          "snr": snrs[name], "frames": counts[name]}
                   for name, _, Z, _ in MIX if name in codes},
           "runs": {}}
    errs = {}
    reps = args.mix_reps
    out["reps_per_run"] = reps
    for key, fn in runs.items():
        fn()  # warm-up: graphs instantiated, workspaces touched
        total = 0.0
        for _ in range(reps):  # the same frames again: a timed region of reps decodes of the mix
            sec, res = fn()
            total += sec
        out["runs"][key], errs[key] = summarise(codes, inputs, counts, total / reps, res)
        out["runs"][key]["timed_seconds"] = total
    for key in runs:
        if key != "per_frame_fp32":
            out["runs"][key]["vs_per_frame_fp32"] = paired(errs["per_frame_fp32"], errs[key])
        if key != "per_code_fp32":
            out["runs"][key]["vs_per_code_fp32"] = paired(errs["per_code_fp32"], errs[key])
    for key in ("multi_fp16", "pools_fp16"):
        out[f"speedup_{key}_vs_per_code_fp32"] = (out["runs"][key]["mbps"]
                                                   / out["runs"]["per_code_fp32"]["mbps"])
    out["speedup_pools_fp16_vs_per_frame_fp32"] = (out["runs"]["pools_fp16"]["mbps"]
                                                   / out["runs"]["per_frame_fp32"]["mbps"])
    emit(out)


# ------------------------------------------------------------------- serve

def serve_once(srv, codes, bank, arrivals, passes):
    """Real-time run of the continuous-batching server on one arrival trace
    (the server is idle before and after). arrivals: list of (t_offset_s,
    code, frame index). Returns latencies, per-request key errors, the run's
    seconds and the number of errors on converged frames (undetected)."""
    results = []
    t0 = time.perf_counter()
    i, N = 0, len(arrivals)
    while i < N or srv.pending():
        now = time.perf_counter() - t0
        while i < N and arrivals[i][0] <= now:
            ta, c, f = arrivals[i]
            llr, syn, _ = bank[c]
            n, wm = codes[c].n, (codes[c].m + 31) // 32
            srv.submit(serve.Request(c, llr[f * n:(f + 1) * n], syn[f * wm:(f + 1) * wm],
                                     tag=(i, c, f), t_arrival=t0 + ta))
            i += 1
        if srv.pending():
            results.extend(srv.tick(passes))
        elif i < N:
            time.sleep(max(0.0, arrivals[i][0] - (time.perf_counter() - t0)))
    t_end = time.perf_counter()
    lat = np.array([r.latency for r in results])
    keys_h = {c: bank[c][2].cpu() for c in codes}
    ordered = sorted(results, key=lambda r: r.tag[0])
    err = np.array([int((r.keys != keys_h[r.code][r.tag[2]]).any()) for r in ordered])
    undetected = int(sum(1 for r, e in zip(ordered, err) if e and r.converged == 1))
    return lat, err, t_end - t0, undetected


def fifo_once(per_frame, bank, max_iter, arrivals):
    """First-in-first-out server decoding one frame at a time with the plain
    FP32 decoder."""
    lat, err = [], []
    t0 = time.perf_counter()
    for ta, c, f in arrivals:
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        llr, syn, key = bank[c]
        d = per_frame.decode(c, llr, syn, f, max_iter)
        err.append(int((d.keys != key[f]).any().item()))  # waits for the decode
        lat.append(time.perf_counter() - t0 - ta)
    return np.array(lat), np.array(err), time.perf_counter() - t0


def trace(rng, rate_fps, N, n_bank, names):
    """N Poisson arrivals at rate_fps, each a uniformly drawn code and frame."""
    t = np.cumsum(rng.exponential(1.0 / rate_fps, N))
    cs = rng.integers(0, len(names), N)
    fs = rng.integers(0, n_bank, N)
    return [(float(t[j]), names[cs[j]], int(fs[j])) for j in range(N)]


def study_serve(args):
    n_bank = 64
    counts = {name: n_bank for name, _, _, _ in MIX}
    codes, bank, snrs = mix_setup(args, counts)
    names = [name for name, _, _, _ in MIX]
    params = q.qcldpc_params_init(msg_format=FMT["fp16"])
    slots = {name: 32 for name in names}
    chunk = 32
    passes = 4
    budget = 64 << 30
    bits = {c: codes[c].n for c in names}
    # capacity: a saturated burst (every request present at t = 0)
    rng = np.random.default_rng(12345)
    burst = [(0.0, names[j % len(names)], int(rng.integers(0, n_bank)))
             for j in range(len(names) * 256)]
    srv = serve.Server(codes, args.max_iter, params, hbm_budget_bytes=budget, chunk_slots=chunk,
                       slots=slots)
    serve_once(srv, codes, bank, burst[:30], passes)  # warm-up: graphs instantiated
    lat, err, sec, _ = serve_once(srv, codes, bank, burst, passes)
    footprint = srv.footprint
    cap_fps = len(burst) / sec
    srv.warm(passes)  # the chunks the burst grew get their step graphs before the sweep
    per_frame = PerFrame(codes)
    fifo_once(per_frame, bank, args.max_iter, burst[:12])  # warm-up of the per-frame decoder
    emit({"study": "serve", "phase": "capacity", "frames": len(burst), "seconds": sec,
          "frames_per_s": cap_fps,
          "mbps": sum(bits[c] for _, c, _ in burst) / sec / 1e6,
          "slots_up_front": slots, "chunk_slots": chunk, "slots_after": srv.slots(),
          "peak_footprint_bytes": srv.peak_used, "passes_per_tick": passes, "msg_format": "fp16",
          "device_footprint_bytes": footprint,
          "mix": {name: {"n": codes[name].n, "snr": snrs[name]} for name in names}})
    for li, load in enumerate(parse_floats(args.loads)):
        arr = trace(np.random.default_rng(1000 + li), load * cap_fps, args.serve_requests, n_bank,
                    names)
        lat, err, sec, undet = serve_once(srv, codes, bank, arr, passes)
        flat, ferr, fsec = fifo_once(per_frame, bank, args.max_iter, arr)
        total_bits = sum(bits[c] for _, c, _ in arr)
        emit({"study": "serve", "load": load, "offered_fps": load * cap_fps, "requests": len(arr),
              "server": {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                         "mbps": total_bits / sec / 1e6, **fer_entry(err),
                         "undetected": undet},
              "per_frame_fifo_fp32": {"p50_ms": 1e3 * float(np.percentile(flat, 50)),
                                      "p99_ms": 1e3 * float(np.percentile(flat, 99)),
                                      "mbps": total_bits / fsec / 1e6, **fer_entry(ferr)},
              "vs_fifo": paired(ferr, err)})


# ---------------------------------------------------------------- schedule

def study_schedule(args):
    """The autotuner on a sample batch of each FER operating point: the time
    each candidate schedule needs to decode the batch, and its choice."""
    F = 16
    for si, item in enumerate(args.fer_points.split(",")):
        cname, snr = item.split(":")
        snr = float(snr)
        mk, Z, label = FER_CODES[cname]
        code = q.create_code_from(mk(Z))
        llr, syn, key = make_frames(code, F, snr, seed=9_000_000 + si)
        lay = q.qcldpc_params_init(schedule=1)
        ws_bytes = q.qcldpc_decode_workspace(code, F, lay)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        wk = (code.k + 31) // 32
        keys = torch.empty(F * wk, dtype=torch.int32, device="cuda")
        conv = torch.empty(F, dtype=torch.int32, device="cuda")
        its = torch.empty(F, dtype=torch.int32, device="cuda")
        best, times = q.qcldpc_autotune(code, llr, syn, F, args.max_iter, None, keys, conv, its,
                                        ws, ws_bytes, reps=3)
        emit({"study": "schedule", "code": f"{label}, Z={Z}, n={code.n}", "snr": snr,
              "frames": F, "max_iter": args.max_iter,
              "ms_per_batch": times,
              "mbps": {k: F * code.n / (v * 1e-3) / 1e6 for k, v in times.items()},
              "chosen": {"schedule": "layered" if best.schedule else "flooding",
                         "layers": best.layers}})


# --------------------------------------------------------------------- et

def study_et(args):
    """Delayed early termination (Sec. IV-A): build the SNR -> et_start table
    from a 16-frame sample per SNR, then decode 64 other frames per SNR with
    the test from iteration 1 and from the table's start."""
    from paper_1702_07740_gb300 import et_lut
    Z = 20000
    code = q.create_code_from(synth.rate002_code(Z))
    wk = (code.k + 31) // 32
    snrs = [0.029, 0.1, 0.13, 0.16, 0.2]
    sample = {}
    for i, snr in enumerate(snrs):
        llr, syn, _ = make_frames(code, 16, snr, seed=9_100_000 + i)
        sample[snr] = (llr, syn, 16)
    lut = et_lut.build(code, sample, args.max_iter)
    del sample
    F = 64
    for i, snr in enumerate(snrs):
        llr, syn, key = make_frames(code, F, snr, seed=9_200_000 + i)
        out = {}
        for name, et in (("test_from_1", 1), ("table", lut.et_start_for(snr))):
            p = q.qcldpc_params_init()
            p.et_start = et
            dec = q.Decoder(code, F, p)
            dec.decode(llr, syn, args.max_iter)  # warm-up: graph instantiation
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dec.decode(llr, syn, args.max_iter)
            e1.record()
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            err = (dec.keys.view(F, wk) != key).any(1).cpu().numpy()
            out[name] = {"et_start": et, "mbps": F * code.n / sec / 1e6,
                         "mean_iters": float(dec.iters.float().mean()),
                         "converged": int(dec.converged.sum()), "errors": int(err.sum()),
                         "keys": dec.keys.clone()}
        same = bool(torch.equal(out["test_from_1"].pop("keys"), out["table"].pop("keys")))
        emit({"study": "et", "code": f"rate 0.02, Z={Z}, n={code.n}", "snr": snr, "frames": F,
              "max_iter": args.max_iter, "same_keys": same, **out})


def run(args):
    torch.cuda.set_device(0)
    q.load()
    {"fer": study_fer, "batch": study_batch, "serve": study_serve,
     "schedule": study_schedule, "et": study_et}[args.study](args)
