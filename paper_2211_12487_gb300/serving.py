"""Continuous-batching serving loop over many TT-ICE* streams on one GPU.

Each client stream (its own shape, batch size and eps) owns one libttice handle whose cores stay
resident on the device.  Increments arrive at any time; a stream has at most one update in flight
(update k+1 needs the cores left by update k), and a fixed pool of slots, each with its own CUDA
stream and host worker thread, runs whichever ready streams come next, so updates of different
streams overlap on the device.  A new stream is admitted only when its projected core memory (the
capacity its handle allocates) fits in the memory budget left by the admitted streams; otherwise it
waits in the admission queue and is admitted as soon as a finished stream releases its memory.
Ranks are not bounded by the method: when an update needs a rank above its handle's capacity, the
capacity is raised in place (device to device) if the grown handle still fits in the budget, and the
update is repeated.

All arithmetic stays in libttice: this module only schedules calls to `ttice_update` (ctypes
releases the GIL during the call, so slots run concurrently).
"""
from __future__ import annotations

import collections
import contextlib
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import torch

from . import ttice as T


@dataclass
class StreamSpec:
    name: str
    dims: tuple
    eps: float
    max_batch: int
    input_dtype: torch.dtype = torch.float32
    precision: str = "fp32"
    max_rank: int = 512


@dataclass
class Request:
    stream: str
    data: torch.Tensor          # device tensor (b, *dims)
    arrival: float = 0.0        # perf_counter time the request became available
    done: float = 0.0
    stats: object = None
    error: Exception | None = None


def default_caps(spec: StreamSpec) -> list[int]:
    """Rank capacities cap_0..cap_d of a new handle: cap_i = min(max_rank, cap_{i-1} n_{i-1})."""
    cap = [1]
    for n in spec.dims:
        cap.append(min(spec.max_rank, cap[-1] * n))
    return cap


def projected_core_bytes(spec: StreamSpec, caps: list[int] | None = None) -> int:
    """Device bytes a handle for `spec` with rank capacities `caps` (default: the creation rule)
    allocates: computed by the library's own creation code in a dry run (ttice_projected_bytes), so
    it is what ttice_device_bytes reports once the handle exists."""
    h = T.ttice_default_heuristics()
    h.precision = T.PRECISIONS[spec.precision]
    h.input_dtype = T.TTICE_F32 if spec.input_dtype == torch.float32 else T.TTICE_F64
    c = T.ttice_default_capacity()
    c.max_batch, c.max_rank = int(spec.max_batch), int(spec.max_rank)
    return T.ttice_projected_bytes(spec.dims, h, c, caps)


class ServingEngine:
    def __init__(self, specs: list[StreamSpec], slots: int = 4, mem_budget: int | None = None,
                 device=None):
        self.device = torch.device(device or "cuda")
        self.specs = {s.name: s for s in specs}
        self.slots = slots
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(free * 0.8)
        self.mem_budget = mem_budget
        self.mem_used = 0
        self.mem_of: dict[str, int] = {}
        self.grow_events = 0  # rank capacities raised after an update needed more
        self.handles: dict[str, T.TTICE] = {}
        self.pending: dict[str, collections.deque] = collections.defaultdict(collections.deque)
        self.busy: set[str] = set()
        self.waiting_admission: collections.deque = collections.deque()
        self.finished_streams: set[str] = set()
        self.failed_streams: dict[str, Exception] = {}  # streams whose handle could not be created
        self.lock = threading.Condition()
        self.ready: queue.Queue = queue.Queue()
        self.completed: list[Request] = []
        self.stop = False
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(slots)]
        for w in self.workers:
            w.start()

    # -------------------------------------------------------------- admission
    def _try_admit(self):
        """Admit waiting streams in arrival order while their projected memory fits."""
        while self.waiting_admission:
            name = self.waiting_admission[0]
            need = projected_core_bytes(self.specs[name])
            if self.mem_used + need > self.mem_budget and self.handles:
                return
            self.waiting_admission.popleft()
            spec = self.specs[name]
            try:
                # an explicit device index is made current for the creation; none: the current one
                ctx = (torch.cuda.device(self.device.index) if self.device.index is not None
                       else contextlib.nullcontext())
                with ctx:
                    h = T.TTICE(spec.dims, spec.eps, precision=spec.precision,
                                input_dtype=spec.input_dtype, max_batch=spec.max_batch,
                                max_rank=spec.max_rank)
            except T.TTICEError as e:
                # the stream cannot be served: its requests complete with the error
                now = time.perf_counter()
                while self.pending[name]:
                    req = self.pending[name].popleft()
                    req.error, req.done = e, now
                    self.completed.append(req)
                self.failed_streams[name] = e
                self.lock.notify_all()
                continue
            self.handles[name] = h
            self.mem_of[name] = h.device_bytes()  # what the handle actually holds
            self.mem_used += self.mem_of[name]
            if self.pending[name]:
                self._schedule(name)

    def _schedule(self, name):
        if name in self.handles and name not in self.busy and self.pending[name]:
            self.busy.add(name)
            self.ready.put(name)

    def submit(self, req: Request):
        with self.lock:
            if not req.arrival:
                req.arrival = time.perf_counter()
            if req.stream in self.failed_streams or req.stream in self.finished_streams:
                # a stream that could not be created, or that its client released, takes no new work
                why = self.failed_streams.get(req.stream) or RuntimeError(f"stream {req.stream} was released")
                req.error, req.done = why, time.perf_counter()
                self.completed.append(req)
                self.lock.notify_all()
                return
            self.pending[req.stream].append(req)
            if req.stream not in self.handles and req.stream not in self.waiting_admission:
                self.waiting_admission.append(req.stream)
                self._try_admit()
            else:
                self._schedule(req.stream)

    def release(self, name: str):
        """The client closed stream `name`: its queued requests complete with an error, an update
        of it that a slot is running is waited for (its handle is never freed under it), then its
        cores are freed and waiting streams admitted.  Later submits to `name` are refused."""
        with self.lock:
            self.finished_streams.add(name)
            now = time.perf_counter()
            gone = RuntimeError(f"stream {name} was released")
            while self.pending[name]:
                req = self.pending[name].popleft()
                req.error, req.done = gone, now
                self.completed.append(req)
            with contextlib.suppress(ValueError):
                self.waiting_admission.remove(name)
            while name in self.busy:  # a slot holds the handle: wait for its update to end
                self.lock.wait(timeout=0.05)
            h = self.handles.pop(name, None)
            if h is not None:
                h.close()
                self.mem_used -= self.mem_of.pop(name, 0)
            self._try_admit()
            self.lock.notify_all()

    # -------------------------------------------------------------- slots
    def _worker(self, slot: int):
        on_gpu = self.device.type == "cuda"
        cuda_stream = torch.cuda.Stream(device=self.device) if on_gpu else None
        while True:
            name = self.ready.get()
            if name is None:
                return
            with self.lock:
                if not self.pending[name] or name not in self.handles:  # cancelled by close()
                    self.busy.discard(name)
                    self.lock.notify_all()
                    continue
                req = self.pending[name].popleft()
                h = self.handles[name]
            try:
                if on_gpu:
                    with torch.cuda.device(self.device), torch.cuda.stream(cuda_stream):
                        cuda_stream.wait_stream(torch.cuda.default_stream(self.device))
                        req.stats = self._update(name, h, req.data, cuda_stream)
                else:  # host-only engine (stand-in handles): no CUDA stream
                    req.stats = self._update(name, h, req.data, None)
            except Exception as e:  # the error is reported with the request
                req.error = e
            req.done = time.perf_counter()
            with self.lock:
                self.completed.append(req)
                self.busy.discard(name)
                self._schedule(name)
                self.lock.notify_all()

    def _update(self, name: str, h: T.TTICE, Y: torch.Tensor, cuda_stream):
        """ttice_update; when the increment needs a rank above its capacity (TTICE_ECAPACITY with the
        rank named), raise that capacity -- to the rank needed, at least doubling it -- if the grown
        handle fits in the memory budget, and repeat the update (a failed update leaves the
        decomposition as it was)."""
        while True:
            try:
                return h.update(Y, stream=cuda_stream)
            except T.TTICEError as e:
                if e.code != T.TTICE_ECAPACITY:
                    raise
                k, need = h.capacity_miss()
                if k == 0:
                    raise
                caps = h.capacities()
                new_caps = list(caps)
                new_caps[k] = max(need, 2 * caps[k])
                grown = projected_core_bytes(self.specs[name], new_caps)
                with self.lock:
                    # the old and the new buffers coexist while the cores are moved
                    if self.mem_used + grown > self.mem_budget:
                        raise
                    self.mem_used += grown
                ok = False
                try:
                    h.reserve_rank(k, new_caps[k])
                    ok = True
                finally:
                    with self.lock:
                        now = h.device_bytes()
                        self.mem_used += now - self.mem_of[name] - grown
                        self.mem_of[name] = now
                        self.grow_events += int(ok)

    def drain(self, timeout: float | None = None) -> bool:
        """Wait until every submitted request has completed."""
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self.lock:
            while any(self.pending[n] for n in self.pending) or self.busy:
                left = None if t_end is None else t_end - time.perf_counter()
                if left is not None and left <= 0:
                    return False
                self.lock.wait(timeout=0.05 if left is None else min(0.05, left))
        return True

    def close(self, cancel_pending: bool = False):
        """Stop the slots.  With cancel_pending, requests not yet started are dropped (the slots
        finish only the updates already running) instead of being run first.  A handle whose slot
        is still inside an update when the wait for the slots ends is not freed under it (it is left
        to the process exit)."""
        if cancel_pending:
            with self.lock:
                for dq in self.pending.values():
                    dq.clear()
        for _ in self.workers:
            self.ready.put(None)
        for w in self.workers:
            w.join(timeout=30)
        with self.lock:
            for name in list(self.handles):
                if name in self.busy:
                    continue
                self.handles.pop(name).close()
                self.mem_used -= self.mem_of.pop(name, 0)

    # -------------------------------------------------------------- reporting
    def latencies_ms(self):
        return sorted((r.done - r.arrival) * 1e3 for r in self.completed if r.error is None)


def percentile(sorted_vals, q):
    if not sorted_vals:
        return float("nan")
    i = min(len(sorted_vals) - 1, max(0, int(math.ceil(q * len(sorted_vals))) - 1))
    return sorted_vals[i]
