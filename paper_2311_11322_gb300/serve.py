"""Continuous batching of independent simulations on one GPU.

Requests (a pile's initial conditions, its parameters and a number of steps)
arrive over time.  The server admits a waiting request as soon as a pile slot
is free and its device footprint (dem_footprint_bytes) fits in the memory
budget, keeps every admitted pile resident in one world, and advances all of
them together: each round is one dem_step call of n steps (n = the smallest
number of steps any resident pile still needs, capped by `chunk`), during
which every pile runs inside the same per-step CUDA graph.  Piles that are done
are read back and removed at the round boundary, freeing slot and memory for
the queue.  Requests arriving while others run are admitted at the next round
boundary, so their work overlaps on the device with the piles already there.

Because every pile's arithmetic is independent of the other piles in the
batch, a request's result is the same alone and in the mix (the GPU tests
check this bit for bit).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    ic: object                 # workloads.PileIC
    params: object             # workloads.Params
    steps: int
    t_arrival: float = 0.0     # seconds after the start of the trace
    # filled by the server
    t_admit: float | None = None
    t_done: float | None = None
    pile: int | None = None
    remaining: int = 0
    status: str = "waiting"    # waiting, running, done, failed
    result: dict = field(default_factory=dict)

    @property
    def n_spheres(self) -> int:
        return int(len(self.ic.radius))

    @property
    def n_agg(self) -> int:
        return int(len(self.ic.counts))


def percentile(xs, q):
    if not xs:
        return None
    return float(np.percentile(np.asarray(xs, float), q))


class Server:
    """Admission by footprint and slots; batched stepping; retirement.

    world: a `dem.World` (or any object with add_pile / step / sync / read /
    remove / piles); footprint: callable (n_spheres, n_agg, K, precision) ->
    bytes; clock: callable returning seconds (wall clock by default).
    """

    def __init__(self, world, footprint, budget_bytes: int, max_piles: int = 64,
                 chunk: int = 200, read_fields=("COM", "VEL", "QUAT", "OMEGA"), clock=None,
                 sleep=None):
        self.world = world
        self.footprint = footprint
        self.budget = int(budget_bytes)
        self.max_piles = int(max_piles)
        self.chunk = int(chunk)
        self.read_fields = tuple(read_fields)
        self.clock = clock or time.perf_counter
        self.sleep = sleep or time.sleep
        self.queue: list[Request] = []
        self.running: dict[int, Request] = {}
        self.done: list[Request] = []
        self.used_bytes = 0
        self.rounds = 0
        self.sphere_steps = 0

    def bytes_of(self, r: Request) -> int:
        return int(self.footprint(r.n_spheres, r.n_agg, int(r.params.max_contacts),
                                  int(r.params.precision)))

    # -------------------------------------------------------------- admission
    def _admit(self, now):
        admitted = []
        still = []
        for r in self.queue:
            if r.t_arrival > now:
                still.append(r)
                continue
            need = self.bytes_of(r)
            if need > self.budget:
                r.status = "failed"
                r.result = {"error": f"footprint {need} B exceeds the budget {self.budget} B"}
                r.t_done = now
                self.done.append(r)
                continue
            if len(self.running) < self.max_piles and self.used_bytes + need <= self.budget:
                r.pile = self.world.add_pile(r.ic, r.params)
                r.t_admit = now
                r.remaining = int(r.steps)
                r.status = "running"
                self.running[r.pile] = r
                self.used_bytes += need
                admitted.append(r)
            else:
                still.append(r)
        self.queue = still
        return admitted

    def _retire(self, now):
        finished = [r for r in self.running.values() if r.remaining <= 0]
        for r in finished:
            for f in self.read_fields:
                r.result[f] = self.world.read(r.pile, f)
            self.world.remove(r.pile)
            del self.running[r.pile]
            self.used_bytes -= self.bytes_of(r)
            r.status = "done"
            r.t_done = now
            self.done.append(r)
        return finished

    # -------------------------------------------------------------- main loop
    def run(self, requests, max_rounds: int | None = None):
        """Serve `requests` (sorted by arrival) until all are done."""
        self.queue = sorted(requests, key=lambda r: r.t_arrival)
        t0 = self.clock()
        while self.queue or self.running:
            now = self.clock() - t0
            self._admit(now)
            if not self.running:
                if not self.queue:
                    break
                nxt = min(r.t_arrival for r in self.queue)
                if nxt > now:
                    self.sleep(nxt - now)
                continue
            n = min(self.chunk, min(r.remaining for r in self.running.values()))
            status = self.world.step(n, check=False)
            self.world.sync(check=False)
            self.rounds += 1
            for r in self.running.values():
                r.remaining -= n
                self.sphere_steps += n * r.n_spheres
            failed = self._failed_piles()
            now = self.clock() - t0
            for pid in failed:
                r = self.running.pop(pid)
                self.world.remove(pid)
                self.used_bytes -= self.bytes_of(r)
                r.status = "failed"
                r.result = {"error": f"pile failed (status {status})"}
                r.t_done = now
                self.done.append(r)
            self._retire(now)
            if max_rounds is not None and self.rounds >= max_rounds:
                break
        return self.stats(self.clock() - t0)

    def _failed_piles(self):
        out = []
        flags = getattr(self.world, "flags", None)
        if flags is None:
            return out
        for pid in list(self.running):
            if flags(pid) & 3:      # slot overflow or non-finite state: the pile is frozen
                out.append(pid)
        return out

    def stats(self, wall):
        ttf = [r.t_done - r.t_arrival for r in self.done if r.status == "done"]
        wait = [r.t_admit - r.t_arrival for r in self.done if r.t_admit is not None]
        return {"requests": len(self.done), "completed": len(ttf),
                "failed": sum(r.status == "failed" for r in self.done),
                "p50_time_to_finish_s": percentile(ttf, 50), "p99_time_to_finish_s": percentile(ttf, 99),
                "p50_queue_wait_s": percentile(wait, 50), "wall_s": wall, "rounds": self.rounds,
                "sphere_steps_per_s": self.sphere_steps / wall if wall > 0 else None}


def trace_requests(trace, make_pile, steps=None):
    """Requests from a workloads.config5_trace list; make_pile(req) -> (ic, params)."""
    out = []
    for k, t in enumerate(trace):
        ic, p = make_pile(t)
        out.append(Request(rid=k, ic=ic, params=p, steps=int(steps or t["steps"]),
                           t_arrival=float(t["t_arrival"])))
    return out
