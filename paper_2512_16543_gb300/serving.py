"""Continuous-batching server for precoder-update requests from many resident beam states.

Each (N, K) class of beam state owns one library handle whose instances are the class's state
slots (G_{t-1} and X = G^{-1} stay resident in the handle's workspace between requests) and a
CUDA stream of its own, so the classes' launches overlap on the device.  A request names a
state and carries that state's next channel H_t.  The server

  * admits states by HBM footprint: a state is given a slot only while the bytes of all
    admitted states (their share of the class workspace plus their input and output rows)
    stay within the budget.  A state that does not fit either is turned away (its requests
    are rejected) or, with admit(..., wait=True), joins a first-come admission queue: its
    requests are held, and it is admitted -- its held requests then join its class's
    pending work -- as soon as retire() frees a slot and the bytes it needs; its requests'
    latency includes that wait;
  * batches continuously: whenever a class has pending requests and fewer than `depth`
    launches in flight, it gathers the pending requests (at most one per state) into the
    class's input rows and launches one masked step for exactly those states -- requests
    that arrive while earlier ones are on the GPU join the next launch, which is queued
    behind the running one on the class's stream (one set of input and output rows per
    launch in flight);
  * runs a state's first request as a masked full inverse and every later one as a masked
    update, so a state's results depend only on its own request sequence: the same alone
    and in any mix (the library's masked steps keep a per-instance snapshot counter).

Latency of a request = completion (its launch's event observed complete) - arrival.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import torch

from . import binding


@dataclass
class Request:
    state: int                   # state id (server-wide)
    H: torch.Tensor              # [K, N] device tensor, this state's next channel
    arrival: float = 0.0         # host time [s]
    done: float | None = None    # host time of completion [s]
    W: torch.Tensor | None = None        # [N, K] result (when keep_results)
    sum_rate: float | None = None


@dataclass
class _Launch:
    event: torch.cuda.Event
    requests: list
    buf: int


@dataclass
class _Class:
    N: int
    K: int
    capacity: int
    handle: binding.WBRZF
    stream: torch.cuda.Stream
    Hbuf: list                   # depth x [capacity, K, N]
    Wbuf: list                   # depth x [capacity, N, K]
    rate: list                   # depth x [capacity] float32
    mask: list                   # depth x [capacity] uint8 (device)
    per_state_bytes: int
    free: list = field(default_factory=list)
    slot_of: dict = field(default_factory=dict)          # state id -> slot
    initialised: set = field(default_factory=set)
    pending: collections.deque = field(default_factory=collections.deque)
    inflight: collections.deque = field(default_factory=collections.deque)
    next_buf: int = 0
    launches: int = 0


class BeamServer:
    """classes: list of (N, K, capacity) or (N, K, capacity, rule); rule: the rank rule of
    every class that names none; budget_bytes: HBM the admitted states may occupy (None:
    unlimited); depth: launches in flight per class."""

    def __init__(self, classes, rule: binding.RankRule | None = None, *, precision="c64",
                 budget_bytes: int | None = None, depth: int = 2, device="cuda",
                 engine: str | None = None, keep_results: bool = False):
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.rule = rule or binding.RankRule()
        self.depth = int(depth)
        self.budget = budget_bytes
        self.keep = keep_results
        self.dtype = torch.complex64 if precision == "c64" else torch.complex128
        self.classes: list[_Class] = []
        self.class_of: dict[int, int] = {}
        self.used_bytes = 0
        self.rejected = 0
        self.completed: list[Request] = []
        self.waiting: collections.deque = collections.deque()   # (state, class, alpha, sigma2)
        self.held: dict[int, list] = {}        # waiting state -> its requests, in order
        self.admitted_after_wait = 0
        for spec in classes:
            N, K, cap = spec[:3]
            crule = spec[3] if len(spec) > 3 else self.rule
            # alpha, sigma2 are per slot; a state's own values are written at admission
            h = binding.WBRZF(cap, N, K, [1.0] * cap, [1.0] * cap, rule=crule,
                              precision=precision, device=self.device,
                              workspace_for="blocked" if K > 64 else "auto")
            if engine is not None:
                h.set_engine(engine)
            st = torch.cuda.Stream(self.device)
            h.set_stream(st)
            esz = 8 if precision == "c64" else 16
            per_state = (h.workspace.numel() // cap +
                         self.depth * (2 * K * N * esz + 4 + 1))   # inputs, outputs, rate, mask
            nb = self.depth                      # one input / output set per launch in flight
            c = _Class(N, K, cap, h, st,
                       [torch.zeros(cap, K, N, dtype=self.dtype, device=self.device)
                        for _ in range(nb)],
                       [torch.zeros(cap, N, K, dtype=self.dtype, device=self.device)
                        for _ in range(nb)],
                       [torch.zeros(cap, dtype=torch.float32, device=self.device)
                        for _ in range(nb)],
                       [torch.zeros(cap, dtype=torch.uint8, device=self.device)
                        for _ in range(nb)],
                       per_state)
            c.free = list(range(cap - 1, -1, -1))
            self.classes.append(c)

    # ------------------------------------------------------------------ admission
    def _fits(self, c: _Class) -> bool:
        return bool(c.free) and (self.budget is None or
                                 self.used_bytes + c.per_state_bytes <= self.budget)

    def _place(self, state: int, cls: int, alpha: float, sigma2: float) -> None:
        c = self.classes[cls]
        slot = c.free.pop()
        c.slot_of[state] = slot
        self.class_of[state] = cls
        self.used_bytes += c.per_state_bytes
        c.handle.set_instance_params(slot, alpha, sigma2, instance_id=state)

    def admit(self, state: int, cls: int, alpha: float, sigma2: float,
              wait: bool = False) -> bool:
        """Give `state` a slot of class `cls` if a slot and the HBM budget allow it; returns
        True when it is admitted now.  With wait=True a state that does not fit joins the
        admission queue instead of being turned away (see retire)."""
        if state in self.class_of or state in self.held:
            raise ValueError(f"state {state} is already admitted or waiting")
        if not self.waiting and self._fits(self.classes[cls]):
            self._place(state, cls, alpha, sigma2)
            return True
        if wait:
            self.waiting.append((state, cls, alpha, sigma2))
            self.held[state] = []
        return False

    def retire(self, state: int) -> None:
        """Free a state's slot (after its requests have completed), then admit waiting states
        in arrival order while the head of the queue fits."""
        cls = self.class_of.pop(state)
        c = self.classes[cls]
        slot = c.slot_of.pop(state)
        c.initialised.discard(state)
        c.free.append(slot)
        self.used_bytes -= c.per_state_bytes
        while self.waiting and self._fits(self.classes[self.waiting[0][1]]):
            st, ci, alpha, sigma2 = self.waiting.popleft()
            self._place(st, ci, alpha, sigma2)
            self.classes[ci].pending.extend(self.held.pop(st))
            self.admitted_after_wait += 1

    # ------------------------------------------------------------------ requests
    def submit(self, req: Request) -> bool:
        """Queue a request; False (counted in `rejected`) for a state that is neither admitted
        nor waiting for admission."""
        cls = self.class_of.get(req.state)
        if cls is None:
            if req.state in self.held:           # waiting for memory: held until admitted
                self.held[req.state].append(req)
                return True
            self.rejected += 1
            return False
        self.classes[cls].pending.append(req)
        return True

    def _launch(self, c: _Class, batch: list, init: bool) -> None:
        b = c.next_buf
        c.next_buf = (b + 1) % self.depth
        with torch.cuda.stream(c.stream):      # temporaries belong to the class's stream
            slots = torch.tensor([c.slot_of[r.state] for r in batch], device=self.device)
            c.Hbuf[b].index_copy_(0, slots, torch.stack([r.H for r in batch]))
            c.mask[b].zero_()
            c.mask[b].index_fill_(0, slots, 1)
        if init:
            c.handle.full_inverse(c.Hbuf[b], c.Wbuf[b], active=c.mask[b])
        else:
            c.handle.update(c.Hbuf[b], c.Wbuf[b], active=c.mask[b])
        c.handle.sum_rate_into(c.rate[b])
        ev = torch.cuda.Event()
        ev.record(c.stream)
        c.inflight.append(_Launch(ev, batch, b))
        c.launches += 1
        for r in batch:
            if init:
                c.initialised.add(r.state)

    def pump(self) -> int:
        """Launch what can be launched, retire completed launches; returns requests done."""
        ndone = 0
        for c in self.classes:
            while c.inflight and c.inflight[0].event.query():
                ln = c.inflight.popleft()
                now = time.perf_counter()
                for r in ln.requests:
                    r.done = now
                    if self.keep:
                        slot = c.slot_of[r.state]
                        r.W = c.Wbuf[ln.buf][slot].clone()
                        r.sum_rate = float(c.rate[ln.buf][slot])
                    self.completed.append(r)
                ndone += len(ln.requests)
            while c.pending and len(c.inflight) < self.depth:
                init, upd, seen, rest = [], [], set(), collections.deque()
                while c.pending:
                    r = c.pending.popleft()
                    if r.state in seen:          # one request per state per launch
                        rest.append(r)
                        continue
                    seen.add(r.state)
                    (upd if r.state in c.initialised else init).append(r)
                if init:                         # first requests: masked full inverse
                    self._launch(c, init, True)
                if upd and len(c.inflight) < self.depth:
                    self._launch(c, upd, False)
                    upd = []
                c.pending = collections.deque(upd) + rest     # not launched: keep their order
        return ndone

    def drain(self) -> None:
        """Run until every admitted state's requests are done (held requests of states still
        waiting for memory stay held)."""
        while any(c.pending or c.inflight for c in self.classes):
            self.pump()

    def close(self) -> None:
        for c in self.classes:
            c.stream.synchronize()
            c.handle.close()

    # ------------------------------------------------------------------ reports
    def latency_ms(self) -> tuple[float, float]:
        lat = sorted(1e3 * (r.done - r.arrival) for r in self.completed)
        if not lat:
            return float("nan"), float("nan")
        p = lambda q: lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))]   # noqa: E731
        return p(0.50), p(0.99)


def poisson_schedule(rate_per_s: float, duration_s: float, n_states: int, seed: int):
    """Open-loop arrivals: (time [s], state id) with exponential gaps at `rate_per_s` and the
    state drawn uniformly."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    n = int(rate_per_s * duration_s * 1.2) + 16
    gaps = torch.empty(n, dtype=torch.float64).exponential_(rate_per_s, generator=g)
    times = torch.cumsum(gaps, 0)
    states = torch.randint(n_states, (n,), generator=g)
    keep = times < duration_s
    return list(zip(times[keep].tolist(), states[keep].tolist()))
