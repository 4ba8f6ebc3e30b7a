#!/usr/bin/env python3
"""Raw decoded throughput of QC-LDPC reverse reconciliation on one or more GB300s.

Workload (the paper-scale case): rate-0.02 QC multi-edge code, 49x50 base,
Z = 20,000 (n = 10^6), 8-D reconciliation LLRs at SNR 0.029, flooding
sum-product with the stop test after every iteration, at most 500 iterations.
One step = the whole hot path over one batch of 16 frames resident in HBM:
qcldpc_llr_8d (8-D map) followed by qcldpc_decode (message passing, stop test,
key bits). Code construction (host tables) happens once, before timing.

Metric: raw decoded Mbit/s = bits of all decoded frames / wall time (the raw
throughput of Sec. IV, timed end to end instead of per iteration). Also
reported: FER (frame error iff the key bits differ from Bob's, Wilson 95 %),
information throughput raw * R * (1 - FER), mean iterations, p50/p99 step
latency. Multi-GPU: independent replicas (frames shard with no exchange),
weak scaling.

``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "rate0.02_n1e6_snr0.029_max500it_16frames"
METRIC = "raw decoded Mbit/s (rate 0.02, n=1e6)"
UNIT = "Mbit/s"
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=16, help="frames per step")
    ap.add_argument("--batches", type=int, default=4, help="distinct batches cycled")
    ap.add_argument("--code", choices=["rate002", "met"], default="rate002",
                    help="rate002: the 49x50 seeded protograph (the headline workload); met: a "
                         "code sampled from the paper's multi-edge distribution (1568x1600, Z=625)")
    ap.add_argument("--Z", type=int, default=20000)
    ap.add_argument("--snr", type=float, default=0.029)
    ap.add_argument("--max-iter", type=int, default=500)
    ap.add_argument("--cpu-iters", type=int, default=12,
                    help="oracle iterations timed for the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reps", type=int, default=20, help="replays per pass for the roofline")
    ap.add_argument("--launch-mode", choices=["graph", "stream"], default="graph",
                    help="stream: host-enqueued passes, for profilers only (not a bench number)")
    ap.add_argument("--msg-format", choices=["fp32", "fp16", "int8"], default="fp32",
                    help="storage of edge messages (arithmetic stays FP32)")
    ap.add_argument("--schedule", choices=["flooding", "layered"], default="flooding")
    ap.add_argument("--vn-pass", choices=["accumulate", "separate"], default="accumulate",
                    help="flooding posteriors: integer sums accumulated by the check pass, or a "
                         "separate variable pass re-reading every message")
    ap.add_argument("--frame-groups", type=int, default=0,
                    help="flooding graph decodes: side-by-side frame groups (0 = library choice, "
                         "1 = one chain)")
    ap.add_argument("--layers", type=int, default=0,
                    help="layered: row groups per iteration (0 = one per base row)")
    ap.add_argument("--study", choices=["fer", "batch", "serve", "schedule", "et"], default=None,
                    help="instead of the throughput line: FER per message format (fer), a "
                         "mixed-rate 256-frame batch (batch) or a serving-load sweep (serve)")
    ap.add_argument("--study-frames", type=int, default=2000, help="fer: frames per SNR")
    ap.add_argument("--fer-formats", default="fp32,fp16,int8",
                    help="fer: message formats to decode (comma-separated, fp32 first)")
    ap.add_argument("--fer-points", default="r002:0.13,r002:0.16,r005:0.5,r010:1.0",
                    help="fer: code:SNR operating points (codes r002, r005, r010 at n = 1e6)")
    ap.add_argument("--mix-snrs", default="0.16,0.5,1.0",
                    help="batch/serve: SNR of the rate 0.02 / 0.05 / 0.10 codes (every length)")
    ap.add_argument("--mix-frames", type=int, default=256, help="batch: frames in the mix")
    ap.add_argument("--mix-reps", type=int, default=20,
                    help="batch: timed decodes of the mix per variant (their mean is reported)")
    ap.add_argument("--loads", default="0.1,0.2,0.3,0.4,0.5,0.6,0.7,0.8,0.9,1.0,1.1,1.2",
                    help="serve: offered load as a fraction of the measured batched capacity")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="serve: Poisson arrivals per load point")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(rank: int, batch: int, frame: int, batches: int, frames: int) -> int:
    """Seed of one frame of one rank: ranks decode disjoint seeded frames
    (replicas, weak scaling; no data is exchanged between ranks)."""
    return synth.frame_seed((rank * batches + batch) * frames + frame)


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the timing rule: the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def wilson(k, n, z=1.96):
    if n == 0:
        return (float("nan"), float("nan"))
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return (max(0.0, c - h), min(1.0, c + h))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


# ------------------------------------------------------------ clock sampler

CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.5)

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 - 0.2 <= r[0] <= self.t1 + 0.2] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v == "Active"})
        sm = [r[1] for r in inside]
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "reasons": reasons, "samples": len(inside)}


# ------------------------------------------------------- algorithmic bytes

def pass_bytes(Z: int, n_h: int, n_d1: int, n_hcols: int, mb: int, msg_bytes: int = 4,
               accumulate: bool = True):
    """Bytes one frame's check-node / variable-node pass must move.

    Check pass: read and write every heavy message (n_h Z messages each way),
    read the degree-1 Phi values (n_d1 Z floats), the heavy posteriors once
    (n_hcols Z floats), the syndrome (mb Z bits) and previous degree-1
    decisions (n_d1 Z bits), write new decisions (n_d1 Z bits).
    Variable pass, separate: read every heavy message once, the heavy channel
    LLRs, and write the heavy posteriors (stored twice, 2 x 4 bytes).
    Variable pass, accumulated: read the two integer partial sums of every
    heavy node and clear them (16 bytes), read its channel LLR and write its
    posterior twice.
    """
    cn = 2 * msg_bytes * n_h * Z + 4 * (n_d1 * Z + n_hcols * Z) + (mb * Z + 2 * n_d1 * Z) / 8
    if accumulate:
        vn = (16 + 4 + 8) * n_hcols * Z
    else:
        vn = msg_bytes * n_h * Z + 4 * 2 * n_hcols * Z
    return cn, vn


def iteration_bytes(Z: int, n_h: int, n_d1: int, n_hcols: int, mb: int, msg_bytes: int = 4):
    """Algorithmic bytes of one flooding iteration of one frame: every heavy
    message read and written once, the degree-1 Phi values read, the heavy
    posteriors read and written with their channel LLRs, the syndrome and the
    degree-1 decisions in and out."""
    return (2 * msg_bytes * n_h * Z + 4 * n_d1 * Z + 12 * n_hcols * Z
            + (mb * Z + 2 * n_d1 * Z) / 8)


def launch_count(group_passes, per_pass: int, unroll: int) -> int:
    """Library kernels one decode step launches: the LLR map, an init and a
    final kernel per frame group, and per_pass kernels for every pass of
    each group's own loop, whose trips run `unroll` passes each (passes
    after the group's frames stopped still launch)."""
    return 1 + 2 * len(group_passes) + sum(-(-p // unroll) * unroll * per_pass for p in group_passes)


def groups_of(args, F):
    """Frame groups the decode runs as (the library's rule for frame_groups:
    by default two for flooding, one chain for layered decoding)."""
    if args.launch_mode != "graph" or F < 2:
        return 1
    return min(args.frame_groups or (2 if args.schedule == "flooding" else 1), F)


def source_hash():
    """Hash of the decoder's kernel sources with comments and blank space
    removed: the committed DRAM counters stay valid across comment edits and
    are dropped once the code itself changes."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1702_07740_gb300", "csrc")
    files = sorted(f for f in os.listdir(csrc)
                   if f.endswith(".cuh") or f == "decode.cu" or f.startswith("check_pass"))
    for f in files:
        with open(os.path.join(csrc, f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(pass_name: str, code: str, msg_format: str, frames: int, schedule: str = "flooding",
                vn_pass: str = "accumulate"):
    """(kernel name, per-launch DRAM bytes) of a decoder pass on a code from
    the committed ncu summary (entries keyed "<code>:<pass>"), or (None,
    None) when the kernel source changed since the capture or the capture was
    of another configuration (code, storage, frames, schedule, posterior
    form)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None, None
    e = d.get(f"{code}:{pass_name}")
    if (not e or e.get("source_hash") != source_hash() or e.get("msg_format", "fp32") != msg_format
            or e.get("frames") != frames or e.get("schedule", "flooding") != schedule
            or e.get("vn_pass", "accumulate") != vn_pass):
        return None, None
    return e.get("kernel"), e.get("dram_bytes_per_launch")


# ------------------------------------------------------------ CPU oracle

def oracle_sample(Z, snr, iters, seed, d=None):
    """Time the FP64 oracle on one frame: 8-D map plus `iters` iterations
    (the rate-0.02 protograph at Z, or the code dict d)."""
    import oracle
    d = synth.rate002_code(Z) if d is None else d
    code = oracle.Code.from_dict(d)
    x, y, bits = synth.channel_frame(code.n, snr, seed)
    m32 = oracle.bob_message(y, bits).astype(np.float32)
    syn = oracle.syndrome(code, bits)
    x64, m64 = x.astype(np.float32).astype(np.float64), m32.astype(np.float64)
    t0 = time.perf_counter()
    q = oracle.llr(x64, m64, snr)
    t1 = time.perf_counter()
    oracle.decode(code, q, syn, iters, et_start=iters + 1)
    t2 = time.perf_counter()
    return code.n, t1 - t0, (t2 - t1) / max(iters, 1)


def oracle_sample_threads(Z, snr, iters, seed, threads, d=None):
    """Time the FP64 oracle on `threads` frames at once, one per host thread
    (the C oracle runs with the interpreter lock released, so the threads
    run on separate cores): each thread maps and decodes its own copy of
    one frame for `iters` iterations. Returns (bits decoded, wall time of
    the maps, wall time per iteration)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    d = synth.rate002_code(Z) if d is None else d
    code = oracle.Code.from_dict(d)
    x, y, bits = synth.channel_frame(code.n, snr, seed)
    m32 = oracle.bob_message(y, bits).astype(np.float32)
    syn = oracle.syndrome(code, bits)
    x64, m64 = x.astype(np.float32).astype(np.float64), m32.astype(np.float64)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        qs = list(ex.map(lambda _: oracle.llr(x64, m64, snr), range(threads)))
        t1 = time.perf_counter()
        list(ex.map(lambda qf: oracle.decode(code, qf, syn, iters, et_start=iters + 1), qs))
        t2 = time.perf_counter()
    return threads * code.n, t1 - t0, (t2 - t1) / max(iters, 1)


def host_cores():
    """Cores this process may run on (the box's nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_rate(n, t_map, t_iter, iters_per_frame):
    """Raw Mbit/s of the oracle, extrapolated to iters_per_frame iterations."""
    return n / (t_map + t_iter * iters_per_frame) / 1e6


# ---------------------------------------------------------------- arms

def run_reference(args, world, rank):
    if rank != 0:
        return
    sample_iters = 2
    cores = host_cores()
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        n, t_map, t_iter = oracle_sample_threads(args.Z, args.snr, sample_iters, synth.frame_seed(s),
                                                 cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append((n, t_map, t_iter, dt))
    t_map = float(np.mean([t[1] for t in times]))
    t_iter = float(np.mean([t[2] for t in times]))
    n = times[0][0]
    value = oracle_rate(n, t_map, t_iter, args.max_iter)
    sample = (f"per step: {cores} frames (n={n // cores}) on {cores} host threads, 8-D map + "
              f"{sample_iters} flooding iterations of the FP64 oracle each, extrapolated to "
              f"{args.max_iter} iterations per frame")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean([t[3] for t in times])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "Z": args.Z, "n": n // cores, "snr": args.snr,
                   "max_iter": args.max_iter},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1702_07740_gb300 import qcldpc as q

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    q.load()
    stream = torch.cuda.current_stream()

    d = synth.rate002_code(args.Z) if args.code == "rate002" else synth.met_code(625)
    code = q.create_code_from(d)
    n, k, F, B = code.n, code.k, args.frames, args.batches
    wm, wk = (code.m + 31) // 32, (k + 31) // 32
    params = q.qcldpc_params_init(launch_mode=1 if args.launch_mode == "stream" else 0,
                                  msg_format={"fp32": 0, "fp16": 1, "int8": 2}[args.msg_format],
                                  schedule=1 if args.schedule == "layered" else 0,
                                  layers=args.layers,
                                  vn_pass=0 if args.vn_pass == "accumulate" else 1,
                                  frame_groups=args.frame_groups)
    layered = args.schedule == "layered"

    # --- seeded inputs, resident in HBM before timing
    host = []
    batches = []
    for b in range(B):
        xs, ys, bs = [], [], []
        for f in range(F):
            seed = replica_seed(rank, b, f, B, F)
            x, y, bits = synth.channel_frame(n, args.snr, seed)
            xs.append(x.astype(np.float32)); ys.append(y.astype(np.float32)); bs.append(bits)
        x_h = torch.from_numpy(np.concatenate(xs)).pin_memory()
        y_d = torch.from_numpy(np.concatenate(ys)).to(dev)
        bits_np = np.stack(bs)
        bits_d = torch.from_numpy(synth.pack_bits(bits_np).view(np.int32).reshape(-1)).to(dev)
        m_d = torch.empty(F * n, dtype=torch.float32, device=dev)
        syn_d = torch.empty(F * wm, dtype=torch.int32, device=dev)
        # Bob's side: public message M = U Y and syndrome s = H C (GPU, untimed)
        q.qcldpc_bob_message_8d(y_d, bits_d, F * n, m_d)
        q.qcldpc_syndrome(code, bits_d, syn_d, F)
        del y_d, bits_d
        batches.append({
            "x": x_h.to(dev), "m": m_d, "syn": syn_d,
            "keys": torch.zeros(F * wk, dtype=torch.int32, device=dev),
            "conv": torch.zeros(F, dtype=torch.int32, device=dev),
            "iters": torch.zeros(F, dtype=torch.int32, device=dev),
        })
        host.append({"x": x_h, "m": m_d.cpu().pin_memory(), "syn": syn_d.cpu().pin_memory(),
                     "key_ref": bits_np[:, :k]})
    torch.cuda.synchronize()
    llr = torch.empty(F * n, dtype=torch.float32, device=dev)
    ws_bytes = q.qcldpc_decode_workspace(code, F, params)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)

    def step(bt):
        q.qcldpc_llr_8d(bt["x"], bt["m"], F * n, args.snr, llr, stream)
        q.qcldpc_decode(code, llr, bt["syn"], F, args.max_iter, params, bt["keys"], bt["conv"],
                        bt["iters"], ws, ws_bytes, stream)

    for s in range(args.warmup):
        step(batches[s % B])
    torch.cuda.synchronize()

    # --- timed region: device-resident inputs
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if sampler:
        sampler.mark(True)
    evs[0].record(stream)
    for s in range(args.steps):
        step(batches[s % B])
        evs[s + 1].record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(False)
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    elapsed = evs[0].elapsed_time(evs[-1]) / 1e3
    if world > 1:
        dist.barrier()
        elapsed = max_over_ranks(elapsed, dev)
    clocks = sampler.stop() if sampler else None
    value = world * args.steps * F * n / elapsed / 1e6

    # --- accuracy and launch count (deterministic: a batch decodes identically each time)
    frame_err = conv_n = 0
    iters_all = []
    # statistics over the batches the timed steps decoded (fewer steps than
    # batches leave some undecoded)
    used = sorted({s % B for s in range(args.steps)})
    G = groups_of(args, F)
    firsts = [g * (F // G) + min(g, F % G) for g in range(G + 1)]  # the library's frame groups
    loop_passes = [0] * B
    group_passes = [[0] * G for _ in range(B)]  # passes each group's own loop needed
    for b in used:
        keys = synth.unpack_bits(batches[b]["keys"].cpu().numpy().view(np.uint32).reshape(F, wk), k)
        conv = batches[b]["conv"].cpu().numpy()
        its = batches[b]["iters"].cpu().numpy()
        frame_err += int((keys != host[b]["key_ref"]).any(axis=1).sum())
        conv_n += int(conv.sum())
        iters_all.extend(its.tolist())
        loop_passes[b] = int(its.max()) + 1
        group_passes[b] = [int(its[firsts[g]:firsts[g + 1]].max()) + 1 for g in range(G)]
    frames_total = len(used) * F
    fer = frame_err / frames_total
    # per step: llr, and per frame group init + final; per loop pass of a
    # group's own loop, check pass + control + variable pass (flooding) or
    # test pass + control + 2 per row group (layered)
    per_pass = 2 + 2 * (args.layers or d["mb"]) if layered else 3
    # each group's loop runs flooding iterations four per trip until its own
    # frames have stopped, and the stream launch mode enqueues max_iter + 1
    # passes; passes after every frame stopped exit at once but still launch
    if args.launch_mode == "stream":
        loop_passes = [args.max_iter + 1] * B
        group_passes = [[args.max_iter + 1] * G for _ in range(B)]
    unroll = 4 if (not layered and args.launch_mode != "stream") else 1
    launches = sum(launch_count(group_passes[s % B], per_pass, unroll) for s in range(args.steps))

    # --- end to end: pinned host inputs -> device -> keys/flags back to host.
    # Two staging buffers and a copy stream: the inputs of step s+1 are copied
    # while step s decodes (every copy still lies inside the timed region).
    stage = [{"x": torch.empty(F * n, dtype=torch.float32, device=dev),
              "m": torch.empty(F * n, dtype=torch.float32, device=dev),
              "syn": torch.empty(F * wm, dtype=torch.int32, device=dev)} for _ in range(2)]
    outs_h = [{"keys": torch.empty(F * wk, dtype=torch.int32).pin_memory(),
               "conv": torch.empty(F, dtype=torch.int32).pin_memory(),
               "iters": torch.empty(F, dtype=torch.int32).pin_memory()} for _ in range(B)]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def prefetch(s, after=None):
        hb, st = host[s % B], stage[s % 2]
        if after is not None:
            copy_stream.wait_event(after)
        copy_stream.wait_event(freed[s % 2])  # step s-2 is done with this buffer
        with torch.cuda.stream(copy_stream):
            st["x"].copy_(hb["x"], non_blocking=True)
            st["m"].copy_(hb["m"], non_blocking=True)
            st["syn"].copy_(hb["syn"], non_blocking=True)
        copied[s % 2].record(copy_stream)

    def e2e_run(s0, steps, start=None):
        prefetch(s0, after=start)
        for s in range(s0, s0 + steps):
            bt, oh, st = batches[s % B], outs_h[s % B], stage[s % 2]
            stream.wait_event(copied[s % 2])
            q.qcldpc_llr_8d(st["x"], st["m"], F * n, args.snr, llr, stream)
            if s + 1 < s0 + steps:
                prefetch(s + 1)
            q.qcldpc_decode(code, llr, st["syn"], F, args.max_iter, params, bt["keys"], bt["conv"],
                            bt["iters"], ws, ws_bytes, stream)
            freed[s % 2].record(stream)
            oh["keys"].copy_(bt["keys"], non_blocking=True)
            oh["conv"].copy_(bt["conv"], non_blocking=True)
            oh["iters"].copy_(bt["iters"], non_blocking=True)

    e2e_run(0, min(args.warmup, 2))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(0, args.steps, start=e0)
    e1.record(stream)
    e1.synchronize()
    e2e_elapsed = e0.elapsed_time(e1) / 1e3
    if world > 1:
        e2e_elapsed = max_over_ranks(e2e_elapsed, dev)
    e2e_value = world * args.steps * F * n / e2e_elapsed / 1e6
    h2d = 2 * F * n * 4 + F * wm * 4
    d2h = F * wk * 4 + 2 * F * 4

    # --- roofline of the dominant pass (replayed with the flooding decode's
    # launch shape; a layered run replays the flooding passes of the same batch)
    rparams = params
    if layered:
        rparams = q.qcldpc_params_init(msg_format=params.msg_format)
        ws_bytes = q.qcldpc_decode_workspace(code, F, rparams)
    q.qcldpc_decode(code, llr, batches[0]["syn"], F, args.max_iter, rparams, batches[0]["keys"],
                    batches[0]["conv"], batches[0]["iters"], ws, ws_bytes, stream)
    cn_ms, vn_ms = q.qcldpc_time_passes(code, F, ws, ws_bytes, args.reps, stream)
    col_count = np.bincount(d["col"], minlength=d["nb"])
    heavy = col_count != 1
    shape = dict(Z=d["Z"], n_h=int(heavy[d["col"]].sum()), n_d1=int((~heavy[d["col"]]).sum()),
                 n_hcols=int(heavy.sum()), mb=d["mb"],
                 msg_bytes={"fp32": 4, "fp16": 2, "int8": 1}[args.msg_format])
    cn_b, vn_b = pass_bytes(**shape, accumulate=args.vn_pass == "accumulate" and not layered)
    it_b = iteration_bytes(**shape)
    peaks, peak_kind = measured_peaks()
    dom, dom_ms, dom_bytes = (("check_pass", cn_ms, cn_b * F) if cn_ms >= vn_ms
                              else ("variable_pass", vn_ms, vn_b * F))
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    kname, traffic = ncu_traffic(dom, args.code, args.msg_format, F, args.schedule, args.vn_pass)
    # device time per loop iteration of the timed decode (its llr, init and
    # final kernels included): the frame groups overlap passes, so this is
    # below the single-kernel replays' cn_ms + vn_ms
    iter_ms = elapsed * 1e3 / sum(loop_passes[s % B] for s in range(args.steps))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # --- CPU oracle baseline (rank 0, one GPU only)
    cpu = None
    mean_iters = float(np.mean(iters_all))
    if world == 1 and not args.no_cpu_baseline:
        nn, t_map, t_iter = oracle_sample(args.Z, args.snr, args.cpu_iters, synth.frame_seed(0), d)
        one = oracle_rate(nn, t_map, t_iter, mean_iters)
        cores = host_cores()
        na, ta_map, ta_iter = oracle_sample_threads(args.Z, args.snr, args.cpu_iters,
                                                    synth.frame_seed(0), cores, d)
        cpu = {"value": oracle_rate(na, ta_map, ta_iter, mean_iters), "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": (f"{cores} frames (n={nn}) on {cores} host threads, one frame each: FP64 "
                          f"8-D map + {args.cpu_iters} flooding iterations, extrapolated to the GPU "
                          f"run's mean {mean_iters:.1f} iterations per frame"),
               "single_core": {"value": one, "cores": 1,
                               "sample": f"1 frame, same map and iterations, one thread"}}

    lo, hi = wilson(frame_err, frames_total)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "msg_format": args.msg_format, "vn_pass": args.vn_pass if not layered else None,
        "frame_groups": groups_of(args, F),
        "schedule": args.schedule if not layered else f"layered, {args.layers or d['mb']} row groups",
        "config": {"workload": WORKLOAD if args.code == "rate002" else
                   "met_rate0.02_n1e6_snr%g_max%dit_%dframes" % (args.snr, args.max_iter, F),
                   "code": args.code, "Z": d["Z"], "n": n, "k": k, "snr": args.snr,
                   "frames_per_step": F, "distinct_frames": frames_total,
                   "max_iter": args.max_iter, "stop_test": "after every iteration",
                   "parallelism": f"replicas x{world}",
                   "l2": "no flush: per-iteration working set "
                         f"{F * (cn_b + vn_b) / 1e6:.0f} MB > 129 MB L2"},
        "fer": fer, "fer_wilson95": [lo, hi], "frames_converged": conv_n,
        "info_mbps": value * (k / n) * (1 - fer), "mean_iters": mean_iters,
        "step_ms_p50": float(np.percentile(step_ms, 50)),
        "step_ms_p99": float(np.percentile(step_ms, 99)),
        # a frame's latency: device time from the start of its step's LLR map
        # to the end of its decode (every frame of a step completes with it)
        "frame_latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                             "p99": float(np.percentile(step_ms, 99)),
                             "frames_per_step": F},
        "iteration_us_per_frame": iter_ms * 1e3 / F,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "copies": "pinned host; inputs double-buffered on a copy stream, step s+1's "
                          "loading while step s decodes"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": kname or dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "cn_ms": cn_ms, "vn_ms": vn_ms,
                     "bytes_per_launch": dom_bytes,
                     # whole flooding iterations of the timed run: algorithmic
                     # bytes of a frame-iteration x frame-iterations per step
                     # / device time per step, of the same peak
                     "iteration_frac": (it_b * F * mean_iters / (elapsed / args.steps) / 1e9 / peak
                                        if not layered else None)},
        "clocks": clocks,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.study:
        import bench_studies
        bench_studies.run(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
