"""Continuous-batching request loop over the library's pools (one pool per code).

A ``Server`` owns one ``Pool`` per code and admits requests by device-memory
footprint: the pools' workspaces are sized at start-up so that their sum fits
the given budget, and a request waits until its code's pool has a free slot.
Each ``tick``:

1. loads waiting requests into free slots (one ``qcldpc_pool_load`` per frame,
   straight from the request's own device buffers);
2. steps every pool by ``passes`` iteration passes in one graph launch
   (``qcldpc_pools_step``), so frames of all codes and all ages share the GPU;
3. reads the slot states of all pools in one device-to-host copy and collects
   each pool's stopped frames in one ``qcldpc_pool_collect``, which frees
   their slots for the next tick.

Host-side scheduling only: all decoding runs in libqcldpc.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import torch

from . import qcldpc as q


@dataclass
class Request:
    code: str
    llr: torch.Tensor        # device float32[n], natural LLRs
    syn: torch.Tensor        # device int32[ceil(m/32)]
    tag: object = None
    t_arrival: float = field(default_factory=time.perf_counter)
    ready: torch.cuda.Event | None = None  # set by submit: the buffers' writes are done


@dataclass
class Result:
    tag: object
    code: str
    keys: torch.Tensor       # host int32[ceil(k/32)] (packed key bits)
    converged: int
    iters: int
    t_arrival: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Server:
    def __init__(self, codes: dict, slots: dict, max_iter: int, params=None,
                 hbm_budget_bytes: int | None = None, stream=None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = params if params is not None else q.qcldpc_params_init()
        need = {name: q.qcldpc_pool_workspace(codes[name], slots[name], self.params) for name in codes}
        if hbm_budget_bytes is not None and sum(need.values()) > hbm_budget_bytes:
            raise ValueError(f"pools need {sum(need.values())} bytes, budget {hbm_budget_bytes}")
        self.codes = codes
        self.pools = {name: q.Pool(codes[name], slots[name], max_iter, self.params, self.stream)
                      for name in codes}
        self.footprint = sum(need.values())
        self.slot_ids = {name: torch.arange(slots[name], dtype=torch.int32, device="cuda")
                         for name in codes}
        self.free = {name: collections.deque(range(slots[name])) for name in codes}
        self.busy = {name: {} for name in codes}   # slot -> Request
        self.queue = {name: collections.deque() for name in codes}
        self.out = {}
        for name, code in codes.items():
            wk = (code.k + 31) // 32
            s = slots[name]
            self.out[name] = (torch.empty((s, wk), dtype=torch.int32, device="cuda"),
                              torch.empty(s, dtype=torch.int32, device="cuda"),
                              torch.empty(s, dtype=torch.int32, device="cuda"))

    def submit(self, req: Request):
        """Queue a request. Its buffers may still be being written on the
        caller's current stream: an event recorded there now orders the
        server's load of them after those writes."""
        req.ready = torch.cuda.Event()
        req.ready.record(torch.cuda.current_stream())
        self.queue[req.code].append(req)

    def pending(self) -> int:
        return sum(len(v) for v in self.queue.values()) + sum(len(v) for v in self.busy.values())

    def tick(self, passes: int = 4) -> list:
        for name, pool in self.pools.items():
            ids = self.slot_ids[name]
            while self.queue[name] and self.free[name]:
                req = self.queue[name].popleft()
                s = self.free[name].popleft()
                if req.ready is not None:
                    self.stream.wait_event(req.ready)
                q.qcldpc_pool_load(pool, 1, ids[s:s + 1], req.llr, req.syn, self.stream)
                self.busy[name][s] = req
        names = [name for name in self.pools if self.busy[name]]
        if not names:
            return []
        q.qcldpc_pools_step([self.pools[name] for name in names], passes, self.stream)
        # one device->host read of every busy pool's slot states (waits for the passes)
        with torch.cuda.stream(self.stream):
            states = torch.cat([self.pools[name].state for name in names]).cpu().tolist()
        now = time.perf_counter()
        done, collected, off = [], [], 0
        for name in names:
            pool = self.pools[name]
            st = states[off: off + pool.n_slots]
            off += pool.n_slots
            stopped = [s for s in self.busy[name] if st[s] == 2]
            if not stopped:
                continue
            keys, conv, iters = self.out[name]
            with torch.cuda.stream(self.stream):
                sel = torch.tensor(stopped, dtype=torch.int32).to(self.slot_ids[name].device)
            n = len(stopped)
            q.qcldpc_pool_collect(pool, n, sel, keys[:n], conv[:n], iters[:n], self.stream)
            collected.append((name, stopped))
        if collected:
            with torch.cuda.stream(self.stream):
                host = {name: tuple(t[:len(stopped)].cpu() for t in self.out[name])
                        for name, stopped in collected}
            for name, stopped in collected:
                k_h, c_h, i_h = host[name]
                for j, s in enumerate(stopped):
                    req = self.busy[name].pop(s)
                    self.free[name].append(s)
                    done.append(Result(req.tag, name, k_h[j].clone(), int(c_h[j]), int(i_h[j]),
                                       req.t_arrival, now))
        return done

    def drain(self, passes: int = 4) -> list:
        out = []
        while self.pending():
            out.extend(self.tick(passes))
        return out
