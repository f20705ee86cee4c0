"""Continuous-batching server of PBD-R scene requests on one GPU.

A request is a scene plus a number of substeps.  The server keeps every
admitted scene resident on the device and runs in ticks; every tick it

1. advances every resident request by one substep in ONE batched pbdr_step
   call, which returns at once (a scene's result does not depend on which
   other scenes share the call, so a request gets the same bytes alone or
   in the mix);
2. while that substep runs on the GPU, admits, first come first served, the
   requests that have arrived, as long as the HBM ledger (an estimate of the
   device bytes per particle against the budget) allows - they join the
   batch from the next tick on;
3. retires the requests that have received all their substeps: reads back
   their final states in one call and destroys their scenes, which frees
   their device ranges for later requests.

Latency of a request = completion time - arrival time (wall clock), where
completion is when its final state has been copied back to the host.  The
tick latency is the device time of one batched substep of all resident
requests (CUDA events around the step on the serving stream).  The host runs
at most one batched substep ahead of the device: before a tick ends it waits
for the previous tick's substep, so admission sees the device's progress.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np

# device bytes held per resident particle (state, rest offsets, neighbour
# lists, scratch and plan buffers), used by the admission ledger
BYTES_PER_PARTICLE = 320


class CudaTimingEvent:
    """A CUDA timing event recorded on a stream given as a torch stream, a
    raw ``cudaStream_t`` value or None (the current stream)."""

    def __init__(self):
        import torch
        self._torch = torch
        self.ev = torch.cuda.Event(enable_timing=True)

    def record(self, stream=None):
        if isinstance(stream, int):
            stream = self._torch.cuda.ExternalStream(stream) if stream else None
        self.ev.record(stream)

    def synchronize(self):
        self.ev.synchronize()

    def elapsed_time(self, end: "CudaTimingEvent") -> float:
        return self.ev.elapsed_time(end.ev)


@dataclasses.dataclass
class Request:
    rid: int
    scene: object
    steps: int
    arrival: float
    admitted: Optional[float] = None
    done: Optional[float] = None
    sid: Optional[int] = None
    due: int = 0               # batched substeps of the server after which it is done


class Server:
    """Continuous batching over a ``binding.Context``-like object.

    ``ctx_factory`` builds the context (a fake one in host-only tests);
    ``clock`` returns seconds (``time.perf_counter`` by default);
    ``event_factory`` returns a timing event with ``record(stream)``,
    ``synchronize()`` and ``elapsed_time(end)`` in ms (CUDA events of the
    serving stream by default; with a fake context and no factory, ticks are
    timed on the host clock).  ``on_result(rid, pos, vel, err_bits)``, if
    given, receives every finished request instead of ``results``: pos and
    vel are views that stay valid only during the call (copy what is kept).
    """

    def __init__(self, hbm_budget_bytes: int = 120 << 30, device: int = 0,
                 ctx_factory: Optional[Callable[[], object]] = None,
                 clock: Callable[[], float] = time.perf_counter, stream=None,
                 bytes_per_particle: int = BYTES_PER_PARTICLE,
                 event_factory: Optional[Callable[[], object]] = None,
                 on_result: Optional[Callable[[int, np.ndarray, np.ndarray, int], None]] = None):
        own_ctx = ctx_factory is None   # the library's own context (a GPU)
        if event_factory is None and own_ctx:
            event_factory = CudaTimingEvent
        if own_ctx:
            from .binding import Context, OPT_AUTOTUNE, OPT_GRAPHS

            def ctx_factory():
                c = Context(device, hbm_budget_bytes)
                # the resident set changes every few ticks: plain launches, no tuning
                c.set_option(OPT_GRAPHS, 0)
                c.set_option(OPT_AUTOTUNE, 0)
                return c
        self.ctx = ctx_factory()
        self.budget = hbm_budget_bytes
        self.bpp = bytes_per_particle
        self.clock = clock
        self.stream = stream
        self.pending: collections.deque = collections.deque()
        self.active: Dict[int, Request] = {}
        self.finished: List[Request] = []
        self.results: Dict[int, tuple] = {}
        self.ledger = 0
        self.event_factory = event_factory
        self.on_result = on_result
        # finished states are read back into page-locked host buffers
        # (grow-only), enqueued on the serving stream between two substeps
        self._pinned = own_ctx
        self._pin_pos = self._pin_vel = self._pin_err = None
        self._inflight: collections.deque = collections.deque()   # (start, end) events per tick
        self.tick_ms: List[float] = []
        self.host_ms = {"admit": 0.0, "step": 0.0, "retire": 0.0}
        self.ticks = 0
        self.work_done = 0            # particle-iterations
        # bookkeeping that changes only on admission and retirement, so a
        # tick costs O(1) host work besides the library calls
        self._stepped = 0             # batched substeps run so far
        self._due: Dict[int, List[Request]] = collections.defaultdict(list)
        self._ids: List[int] = []     # scene handles of the resident requests
        self._ids_dirty = False
        self._tick_work = 0           # particle-iterations of one batched substep
        self._next = 0
        self.t0 = None

    # ---- requests ----------------------------------------------------------
    def submit(self, scene, steps: int, arrival: float = 0.0) -> int:
        """Queues a request (arrival in seconds from the start of run())."""
        if steps < 1:
            raise ValueError("a request needs at least one substep")
        rid = self._next
        self._next += 1
        self.pending.append(Request(rid, scene, int(steps), float(arrival)))
        return rid

    def _cost(self, req: Request) -> int:
        return self.bpp * int(req.scene.num_particles)

    def _admit(self, now: float) -> int:
        n = 0
        while self.pending and self.pending[0].arrival <= now:
            req = self.pending[0]
            cost = self._cost(req)
            if self.active and self.ledger + cost > self.budget:
                break                  # wait for memory to free up (FIFO: no overtaking)
            try:
                sid = self.ctx.create_scene(req.scene)
            except RuntimeError as e:  # the library's own budget check
                if getattr(e, "code", None) == -3 and self.active:
                    break
                raise
            self.pending.popleft()
            req.sid = sid
            req.admitted = now
            req.due = self._stepped + req.steps     # it joins the next batched substep
            self._due[req.due].append(req)
            self._tick_work += int(req.scene.num_particles) * int(req.scene.iterations)
            self._ids_dirty = True
            self.ledger += cost
            self.active[req.rid] = req
            n += 1
        return n

    def _take_done(self) -> List[Request]:
        """Removes the requests that the last batched substep finished from
        the resident set (they take no further substep)."""
        done = self._due.pop(self._stepped, [])   # in admission order
        for req in done:
            self._tick_work -= int(req.scene.num_particles) * int(req.scene.iterations)
            del self.active[req.rid]
            self._ids_dirty = True
        return done

    def _read_async(self, done: List[Request]):
        """Enqueues the read of finished requests on the serving stream, after
        the substep that finished them and before the next one (no kernel of
        the next substep competes with it); returns (pos, vel, err, event) or
        None where reads are synchronous (a context without asynchronous
        reads, or no timing events)."""
        if not (done and self._pinned and self.event_factory is not None):
            return None
        import torch
        total = sum(int(r.scene.num_particles) for r in done)
        if self._pin_pos is None or self._pin_pos.shape[0] < total:
            cap = max(total, 2 * (0 if self._pin_pos is None else self._pin_pos.shape[0]))
            self._pin_pos = torch.empty((cap, 3), dtype=torch.float32, pin_memory=True).numpy()
            self._pin_vel = torch.empty((cap, 3), dtype=torch.float32, pin_memory=True).numpy()
        if self._pin_err is None or self._pin_err.shape[0] < len(done):
            cap = max(len(done), 2 * (0 if self._pin_err is None else self._pin_err.shape[0]))
            self._pin_err = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        pos, vel, err = self._pin_pos[:total], self._pin_vel[:total], self._pin_err[:len(done)]
        self.ctx.read_states_async([r.sid for r in done], pos, vel, err, stream=self.stream)
        ev = self.event_factory()
        ev.record(self.stream)
        return pos, vel, err, ev

    def _retire(self, done: List[Request], read=None):
        """Delivers and frees finished requests: waits for their enqueued
        read (`read` from _read_async), or reads them synchronously."""
        if not done:
            return
        if read is not None:
            pos, vel, err, ev = read
            ev.synchronize()
        else:
            pos, vel, err = self.ctx.read_states([r.sid for r in done], stream=self.stream)
        now = self.clock() - self.t0              # the results are on the host now
        at = 0
        for k, req in enumerate(done):
            n = int(req.scene.num_particles)
            if self.on_result is not None:
                self.on_result(req.rid, pos[at:at + n], vel[at:at + n], int(err[k]))
            else:
                self.results[req.rid] = (pos[at:at + n].copy(), vel[at:at + n].copy(), int(err[k]))
            at += n
            self.ctx.destroy_scene(req.sid)
            self.ledger -= self._cost(req)
            req.done = now
            self.finished.append(req)

    # ---- main loop -----------------------------------------------------------
    def _drain(self, keep: int):
        """Waits until at most `keep` batched substeps are in flight and
        records the device time of the finished ones."""
        while len(self._inflight) > keep:
            ev0, ev1 = self._inflight.popleft()
            ev1.synchronize()
            self.tick_ms.append(float(ev0.elapsed_time(ev1)))

    def tick(self) -> bool:
        """One batched substep + retirement + admission round; False when idle.

        The requests the previous substep finished leave the resident set
        first and their read is enqueued, then the next substep (both
        asynchronous, on the serving stream); only then does the host wait
        for the read, deliver and free them and admit new requests, so that
        host work overlaps the substep on the device."""
        t_0 = self.clock()
        done = self._take_done()
        read = self._read_async(done)
        stepped = bool(self.active)
        if stepped:
            if self._ids_dirty:
                self._ids = [r.sid for r in self.active.values()]
                self._ids_dirty = False
            if self.event_factory is not None:
                ev0, ev1 = self.event_factory(), self.event_factory()
                ev0.record(self.stream)
                self.ctx.step(self._ids, 1, self.stream)   # asynchronous
                ev1.record(self.stream)
                self._inflight.append((ev0, ev1))
            else:
                self.ctx.step(self._ids, 1, self.stream)
            self._stepped += 1
            self.work_done += self._tick_work
        t_a = self.clock()
        self._retire(done, read)                   # waits for the read only
        t_b = self.clock()
        self._admit(t_b - self.t0)                 # host work overlaps the substep
        self._drain(keep=1)                        # at most one substep ahead of the device
        t_c = self.clock()
        if not stepped:
            return bool(self.pending or self.active)
        self.host_ms["step"] += (t_a - t_0) * 1e3
        self.host_ms["retire"] += (t_b - t_a) * 1e3
        self.host_ms["admit"] += (t_c - t_b) * 1e3
        if self.event_factory is None:
            self.tick_ms.append((t_c - t_0) * 1e3)
        self.ticks += 1
        return True

    def run(self, realtime: bool = True, max_ticks: Optional[int] = None) -> dict:
        """Serves until every submitted request is finished.  With realtime
        the arrival times are honoured against the wall clock (idle gaps are
        slept through); otherwise every request counts as arrived."""
        self.t0 = self.clock()
        if not realtime:
            for r in self.pending:
                r.arrival = 0.0
        while self.pending or self.active:
            if max_ticks is not None and self.ticks >= max_ticks:
                break
            if not self.active and self.pending:
                wait = self.pending[0].arrival - (self.clock() - self.t0)
                if wait > 0:
                    if realtime:
                        time.sleep(min(wait, 0.05))
                    continue
            self.tick()
        self._drain(keep=0)
        return self.stats()

    def stats(self) -> dict:
        lat = np.array([(r.done - r.arrival) * 1e3 for r in self.finished]) if self.finished else np.zeros(0)
        tk = np.array(self.tick_ms) if self.tick_ms else np.zeros(0)
        wall = (self.clock() - self.t0) if self.t0 is not None else 0.0

        def pct(a, q):
            return float(np.percentile(a, q)) if a.size else None
        return {
            "requests": len(self.finished), "ticks": self.ticks, "wall_s": wall,
            "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
            "tick_ms_p50": pct(tk, 50), "tick_ms_p99": pct(tk, 99),
            "particle_iters": self.work_done,
            "host_ms_per_tick": {k: v / max(self.ticks, 1) for k, v in self.host_ms.items()},
            "achieved_particle_iters_per_s": self.work_done / wall if wall > 0 else None,
        }


def poisson_trace(rate_hz: float, duration_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate (seeded)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.array(out)
        out.append(t)
