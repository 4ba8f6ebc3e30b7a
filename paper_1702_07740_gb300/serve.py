"""Continuous-batching request loop over the library's pools.

A ``Server`` admits each request against one device-memory budget shared by
all codes. Frame state lives in pool chunks: a chunk is a ``Pool`` of slots of
one code, and a code holds as many chunks as its requests need. A code's
first chunk has ``chunk_slots`` slots and each further one twice as many as
the previous (at most ``max_chunk_slots``), so a busy code holds a few large
chunks rather than many small ones. A request is admitted when its code has a free slot, or when
one more chunk of its code fits the budget; if the budget is full, chunks
with no frame in them (of any code) are released first. So memory that one
code no longer uses goes to another, and a request waits only while every
byte of the budget holds running frames. Waiting requests are scanned in
arrival order, and one that cannot be placed does not hold back later
requests of codes that have room.

Each ``tick``:

1. admits waiting requests (one ``qcldpc_pool_load`` per frame, straight from
   the request's own device buffers, ordered after the writes that produced
   them);
2. steps every chunk that holds frames by ``passes`` iteration passes, each
   chunk with its own cached step graph (``qcldpc_pool_step``) on one of a
   few side streams, so frames of all codes and all ages share the GPU and no
   graph is rebuilt when the set of busy chunks changes;
3. reads the slot states of those chunks in one device-to-host copy and
   collects each chunk's stopped frames in one ``qcldpc_pool_collect``, which
   frees their slots for the next tick.

Chunks that stay empty for ``idle_seconds`` are released as well (and
created again when their code needs them, which costs a workspace
allocation and a graph instantiation; ``warm`` instantiates the step graphs
of the chunks a server holds). Host-side scheduling only: all
decoding runs in libqcldpc.
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


class _Chunk:
    """One pool of a code with its slot bookkeeping and output buffers."""

    def __init__(self, name, code, n_slots, max_iter, params, stream):
        self.name, self.n_slots = name, n_slots
        self.pool = q.Pool(code, n_slots, max_iter, params, stream)
        self.bytes = self.pool.ws_bytes
        self.slot_ids = torch.arange(n_slots, dtype=torch.int32, device="cuda")
        self.free = collections.deque(range(n_slots))
        self.busy = {}           # slot -> Request
        self.idle_since = time.perf_counter()  # when the chunk last became empty
        wk = (code.k + 31) // 32
        self.out = (torch.empty((n_slots, wk), dtype=torch.int32, device="cuda"),
                    torch.empty(n_slots, dtype=torch.int32, device="cuda"),
                    torch.empty(n_slots, dtype=torch.int32, device="cuda"))


class Server:
    """codes: name -> Code. hbm_budget_bytes caps the sum of the chunks' pool
    workspaces (None: no cap). chunk_slots: slots of a code's first chunk,
    the smallest unit in which its frame state grows and shrinks; later
    chunks double up to max_chunk_slots. slots (optional): name -> slots to
    allocate up front."""

    def __init__(self, codes: dict, max_iter: int, params=None, hbm_budget_bytes: int | None = None,
                 chunk_slots: int = 16, slots: dict | None = None, idle_seconds: float = 30.0,
                 stream=None, n_streams: int = 8, max_chunk_slots: int = 512):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.side = [torch.cuda.Stream() for _ in range(n_streams)]
        self.params = params if params is not None else q.qcldpc_params_init()
        self.codes, self.max_iter = codes, max_iter
        self.budget = hbm_budget_bytes
        self.chunk_slots, self.max_chunk_slots, self.idle_seconds = chunk_slots, max_chunk_slots, idle_seconds
        self.chunk_bytes = {name: q.qcldpc_pool_workspace(codes[name], chunk_slots, self.params)
                            for name in codes}
        if self.budget is not None and min(self.chunk_bytes.values()) > self.budget:
            raise ValueError(f"no chunk fits the budget of {self.budget} bytes")
        self.chunks = {name: [] for name in codes}
        self.used = 0
        self.peak_used = 0
        self.queue = collections.deque()
        for name, s in (slots or {}).items():
            while sum(ch.n_slots for ch in self.chunks[name]) < s:
                if not self._grow(name):
                    raise ValueError(f"initial slots of {name} exceed the budget")

    # ------------------------------------------------------------ memory

    @property
    def footprint(self) -> int:
        """Bytes of device memory the chunks hold now."""
        return self.used

    def _next_slots(self, name) -> int:
        return min(self.max_chunk_slots, self.chunk_slots << len(self.chunks[name]))

    def _grow(self, name, n_slots: int | None = None) -> _Chunk | None:
        n_slots = n_slots or self._next_slots(name)
        need = q.qcldpc_pool_workspace(self.codes[name], n_slots, self.params)
        if self.budget is not None and self.used + need > self.budget:
            return None
        with torch.cuda.stream(self.stream):
            ch = _Chunk(name, self.codes[name], n_slots, self.max_iter, self.params, self.stream)
        self.chunks[name].append(ch)
        self.used += ch.bytes
        self.peak_used = max(self.peak_used, self.used)
        return ch

    def _release(self, ch: _Chunk):
        # the server's stream is idle here: every tick ends with a blocking
        # read of its results
        self.chunks[ch.name].remove(ch)
        self.used -= ch.bytes
        del ch.pool

    def _reclaim(self, need: int) -> bool:
        """Release empty chunks, longest idle first, until `need` more bytes
        fit the budget."""
        empty = sorted((ch for cs in self.chunks.values() for ch in cs if not ch.busy),
                       key=lambda ch: ch.idle_since)
        for ch in empty:
            if self.used + need <= self.budget:
                break
            self._release(ch)
        return self.used + need <= self.budget

    def _place(self, name):
        for ch in self.chunks[name]:
            if ch.free:
                return ch
        # the next (doubled) chunk if it fits, else the smallest one, after
        # releasing empty chunks if the budget needs it
        ch = self._grow(name) or self._grow(name, self.chunk_slots)
        if ch is None and self._reclaim(self.chunk_bytes[name]):
            ch = self._grow(name, self.chunk_slots)
        return ch

    # ------------------------------------------------------------ requests

    def submit(self, req: Request):
        """Queue a request. Its buffers may still be being written on the
        caller's current stream: an event recorded there now orders the
        server's load of them after those writes."""
        req.ready = torch.cuda.Event()
        req.ready.record(torch.cuda.current_stream())
        self.queue.append(req)

    def pending(self) -> int:
        return len(self.queue) + sum(len(ch.busy) for cs in self.chunks.values() for ch in cs)

    def slots(self) -> dict:
        """Slots each code holds now."""
        return {name: sum(ch.n_slots for ch in cs) for name, cs in self.chunks.items()}

    def _admit(self):
        waiting = collections.deque()
        full = set()  # codes that found no room this tick
        while self.queue:
            req = self.queue.popleft()
            ch = None if req.code in full else self._place(req.code)
            if ch is None:
                full.add(req.code)
                waiting.append(req)
                continue
            s = ch.free.popleft()
            if req.ready is not None:
                self.stream.wait_event(req.ready)
            q.qcldpc_pool_load(ch.pool, 1, ch.slot_ids[s:s + 1], req.llr, req.syn, self.stream)
            ch.busy[s] = req
        self.queue = waiting

    def tick(self, passes: int = 4) -> list:
        self._admit()
        live = [ch for cs in self.chunks.values() for ch in cs if ch.busy]
        now = time.perf_counter()
        for cs in self.chunks.values():
            for ch in list(cs):
                if not ch.busy and now - ch.idle_since >= self.idle_seconds:
                    self._release(ch)
        if not live:
            return []
        # fork: chunk i steps on side stream i mod n after this tick's loads,
        # with its own cached graph; join before the states are read
        start = torch.cuda.Event()
        start.record(self.stream)
        used = self.side[: min(len(self.side), len(live))]
        for st in used:
            st.wait_event(start)
        for i, ch in enumerate(live):
            q.qcldpc_pool_step(ch.pool, passes, used[i % len(used)])
        for st in used:
            ev = torch.cuda.Event()
            ev.record(st)
            self.stream.wait_event(ev)
        # one device->host read of every stepped chunk's slot states (waits for the passes)
        with torch.cuda.stream(self.stream):
            states = torch.cat([ch.pool.state for ch in live]).cpu().tolist()
        now = time.perf_counter()
        done, collected, off = [], [], 0
        for ch in live:
            st = states[off: off + ch.n_slots]
            off += ch.n_slots
            stopped = [s for s in ch.busy if st[s] == 2]
            if not stopped:
                continue
            keys, conv, iters = ch.out
            with torch.cuda.stream(self.stream):
                sel = torch.tensor(stopped, dtype=torch.int32).to(ch.slot_ids.device)
            n = len(stopped)
            q.qcldpc_pool_collect(ch.pool, n, sel, keys[:n], conv[:n], iters[:n], self.stream)
            collected.append((ch, stopped))
        if collected:
            with torch.cuda.stream(self.stream):
                host = [tuple(t[:len(stopped)].cpu() for t in ch.out) for ch, stopped in collected]
            for (ch, stopped), (k_h, c_h, i_h) in zip(collected, host):
                for j, s in enumerate(stopped):
                    req = ch.busy.pop(s)
                    ch.free.append(s)
                    if not ch.busy:
                        ch.idle_since = now
                    done.append(Result(req.tag, ch.name, k_h[j].clone(), int(c_h[j]), int(i_h[j]),
                                       req.t_arrival, now))
        return done

    def warm(self, passes: int = 4):
        """Instantiate the step graph of every chunk for `passes` (a step of
        an empty chunk exits at once)."""
        for cs in self.chunks.values():
            for ch in cs:
                q.qcldpc_pool_step(ch.pool, passes, self.stream)
        self.stream.synchronize()

    def drain(self, passes: int = 4) -> list:
        out = []
        while self.pending():
            out.extend(self.tick(passes))
        return out
