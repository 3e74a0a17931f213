"""Continuous-batching server for parallel-tempering jobs.

Requests (one PT problem each: L, betas, J, h, seed, sweeps, exchange interval) arrive over
time. The server:

* admits waiting requests in arrival order while their device state fits the HBM budget
  (the library's own estimate, `pt_estimate_device_bytes`); an admitted request's lattice
  is created on the device and stays there until it finishes;
* every tick advances all resident requests together by min(slice, remaining) sweeps in one
  `pt_sweep_batch` call -- requests admitted while others run join the next tick, so their
  work overlaps on the GPU;
* reads the results of finished requests (energies, magnetisations, temperature map, swap
  counters), frees their state and budget, and records latency = completion - arrival.

Because exchanges follow the global sweep count of each problem, running a request in
slices inside a changing mix gives exactly the result of running it alone.

The device work goes through an `Engine`; `LibEngine` is libpt. Tests of the scheduling
logic substitute a fake engine and run without a GPU.
"""
from __future__ import annotations

import dataclasses
import heapq
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from .workloads import Problem, Request


@dataclasses.dataclass
class Result:
    rid: int
    problem: Problem
    arrival: float
    admitted: float
    finished: float
    E_int: np.ndarray
    M: np.ndarray
    scale: int
    slot_of_temp: np.ndarray
    attempted: np.ndarray
    accepted: np.ndarray

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def energies(self) -> np.ndarray:
        return self.E_int.astype(np.float64) / self.scale


class Engine:
    """What the server needs from the device side."""

    def estimate_bytes(self, p: Problem) -> int:
        raise NotImplementedError

    def create(self, p: Problem):
        raise NotImplementedError

    def advance(self, handles: Sequence, n: Sequence[int], every: Sequence[int]) -> None:
        raise NotImplementedError

    def read(self, handle) -> dict:
        raise NotImplementedError

    def read_many(self, handles: Sequence) -> List[dict]:
        """read() of several problems; an engine may do it in one transfer."""
        return [self.read(h) for h in handles]

    def destroy(self, handle) -> None:
        raise NotImplementedError

    def synchronize(self) -> None:
        pass


class LibEngine(Engine):
    """libpt on the current CUDA device; every problem runs on one torch stream."""

    def __init__(self, stream=None, use_torch_allocator: bool = True):
        import torch

        from . import api
        self.api = api
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        if use_torch_allocator:
            api.use_torch_allocator(True)

    def estimate_bytes(self, p: Problem) -> int:
        return self.api.estimate_device_bytes(p.L, p.betas, p.J, p.h)

    def create(self, p: Problem):
        return self.api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=self.stream)

    def advance(self, handles, n, every):
        self.api.sweep_batch(handles, n, every)

    def read(self, h) -> dict:
        E = h.energies_int()
        M = h.magnetisations()
        att, acc = h.swap_stats()
        return dict(E_int=E, M=M, scale=h.scale, slot_of_temp=h.chain_map(), attempted=att,
                    accepted=acc)

    def read_many(self, handles) -> List[dict]:
        # one energy-count launch, one gather and one copy for all of them (pt_read_batch)
        recs = self.api.read_batch(list(handles))
        return [dict(E_int=r["E_int"], M=r["M"], scale=h.scale, slot_of_temp=r["chain_map"],
                     attempted=r["attempted"], accepted=r["accepted"])
                for h, r in zip(handles, recs)]

    def destroy(self, h) -> None:
        h.close()

    def synchronize(self) -> None:
        self.stream.synchronize()


@dataclasses.dataclass
class _Active:
    req: Request
    handle: object
    nbytes: int
    admitted: float
    done: int = 0


class Server:
    """Admission by device-memory budget plus continuous batching in slices of sweeps."""

    def __init__(self, engine: Engine, budget_bytes: int = 80 * 10 ** 9, slice_sweeps: int = 100,
                 max_active: int = 4096, clock: Callable[[], float] = time.perf_counter):
        if budget_bytes <= 0 or slice_sweeps <= 0 or max_active <= 0:
            raise ValueError("budget, slice and max_active must be positive")
        self.engine = engine
        self.budget = int(budget_bytes)
        self.slice = int(slice_sweeps)
        self.max_active = int(max_active)
        self.clock = clock
        self.used = 0
        self.peak_used = 0
        self.waiting: List = []  # heap of (arrival, rid, request, estimated bytes)
        self.active: List[_Active] = []
        self.results: Dict[int, Result] = {}
        self.rejected: Dict[int, str] = {}
        self.ticks = 0
        self.t0 = None
        self.attempts_done = 0.0
        self.realtime = True

    # -- intake -----------------------------------------------------------------------------
    def submit(self, req: Request) -> None:
        nbytes = int(self.engine.estimate_bytes(req.problem))
        if nbytes <= 0:
            self.rejected[req.rid] = "invalid problem"
            return
        if nbytes > self.budget:
            self.rejected[req.rid] = "needs %d bytes, more than the whole budget" % nbytes
            return
        heapq.heappush(self.waiting, (req.arrival, req.rid, req, nbytes))

    def cancel(self, rid: int) -> bool:
        """Drop a waiting or running request; its memory returns to the budget."""
        for k, (_, r, _, _) in enumerate(self.waiting):
            if r == rid:
                self.waiting.pop(k)
                heapq.heapify(self.waiting)
                self.rejected[rid] = "cancelled"
                return True
        for k, a in enumerate(self.active):
            if a.req.rid == rid:
                self.engine.destroy(a.handle)
                self.used -= a.nbytes
                self.active.pop(k)
                self.rejected[rid] = "cancelled"
                return True
        return False

    # -- one scheduling step -----------------------------------------------------------------
    def _now(self) -> float:
        return self.clock() - self.t0

    def _admit(self, now: float) -> int:
        n = 0
        while self.waiting and len(self.active) < self.max_active:
            arrival, rid, req, nbytes = self.waiting[0]
            if (self.realtime and arrival > now) or self.used + nbytes > self.budget:
                break  # arrival order: nobody overtakes the head of the queue
            heapq.heappop(self.waiting)
            try:
                h = self.engine.create(req.problem)
            except Exception as exc:  # allocation failure and the like: the request fails
                self.rejected[rid] = "create failed: %s" % exc
                continue
            self.used += nbytes
            self.peak_used = max(self.peak_used, self.used)
            self.active.append(_Active(req=req, handle=h, nbytes=nbytes, admitted=now))
            n += 1
        return n

    def step(self) -> int:
        """Admit, advance every resident request by one slice, retire finished ones.
        Returns the number of requests retired."""
        if self.t0 is None:
            self.t0 = self.clock()
        self._admit(self._now())
        if not self.active:
            return 0
        n = [min(self.slice, a.req.problem.sweeps - a.done) for a in self.active]
        every = [a.req.problem.every for a in self.active]
        self.engine.advance([a.handle for a in self.active], n, every)
        for a, k in zip(self.active, n):
            p = a.req.problem
            a.done += k
            self.attempts_done += float(p.L * p.L * p.R) * k
        self.ticks += 1
        finished = [a for a in self.active if a.done >= a.req.problem.sweeps]
        if not finished:
            return 0
        self.active = [a for a in self.active if a.done < a.req.problem.sweeps]
        # the finished requests' results in one read (it synchronises the problems' stream)
        datas = self.engine.read_many([a.handle for a in finished])
        now = self._now()
        for a, data in zip(finished, datas):
            self.results[a.req.rid] = Result(rid=a.req.rid, problem=a.req.problem,
                                             arrival=a.req.arrival, admitted=a.admitted,
                                             finished=now, **data)
            self.engine.destroy(a.handle)
            self.used -= a.nbytes
        return len(finished)

    def idle(self) -> bool:
        return not self.active

    def run(self, requests: Sequence[Request], realtime: bool = True,
            timeout_s: Optional[float] = None) -> Dict[int, Result]:
        """Serve a request stream: request r becomes visible at r.arrival seconds after the
        start (at once when realtime is False). Returns the results by request id."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        self.realtime = realtime
        self.t0 = self.clock()
        k = 0
        while k < len(pending) or self.waiting or self.active:
            now = self._now()
            while k < len(pending) and (not realtime or pending[k].arrival <= now):
                self.submit(pending[k])
                k += 1
            if not self.active and not self.waiting:
                if k < len(pending):  # nothing to do until the next arrival
                    time.sleep(max(0.0, min(0.002, pending[k].arrival - now)))
                continue
            self.step()
            if timeout_s is not None and self._now() > timeout_s:
                raise TimeoutError("serving did not finish within %.1f s" % timeout_s)
        self.engine.synchronize()
        return self.results

    # -- report ------------------------------------------------------------------------------
    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.results.values()])
        wall = max((r.finished for r in self.results.values()), default=0.0)
        return {
            "requests": len(self.results), "rejected": len(self.rejected),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_s": float(lat.mean()) if lat.size else None,
            "attempts": self.attempts_done,
            "wall_s": wall,
            "attempts_per_s": self.attempts_done / wall if wall > 0 else None,
            "ticks": self.ticks, "peak_bytes": self.peak_used, "budget_bytes": self.budget,
        }


def mean_attempts(requests: Sequence[Request]) -> float:
    return float(np.mean([r.problem.attempts for r in requests]))


def bench_serve(args, rank, world, stream):
    """bench.py --workload serve: the Poisson request stream at about 80% of the batched
    throughput measured just before, on one GPU."""
    import torch

    from . import autotune
    from . import workloads as W
    # the launch shape tuned for this request mix (the batched workload's may differ); the
    # caller's shape is put back at the end
    before = autotune.get_tuning()
    autotune.apply_cached_or_default("serve")
    try:
        return _bench_serve(args, stream)
    finally:
        autotune.set_tuning(**before)


def _bench_serve(args, stream):
    import torch

    from . import workloads as W
    eng = LibEngine(stream=stream)
    # the service rate: batched throughput on a sample of the same request mix
    probe = W.serving_requests(n=64, rate_per_s=1.0, draw_seed=4242)
    hs = [eng.create(r.problem) for r in probe]
    # one short untimed call first: the first batch call of a process also sets up the
    # library's side streams and the launch attributes
    eng.advance(hs, [1] * len(hs), [1] * len(hs))
    torch.cuda.synchronize()
    n = [min(200, r.problem.sweeps) for r in probe]
    t0 = time.perf_counter()
    eng.advance(hs, n, [1] * len(hs))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    peak = sum(r.problem.L ** 2 * r.problem.R * k for r, k in zip(probe, n)) / dt
    for h in hs:
        eng.destroy(h)
    nreq = getattr(args, "requests", 2000)
    base = W.serving_requests(n=nreq, rate_per_s=1.0)
    rate = 0.8 * peak / mean_attempts(base)
    reqs = W.serving_requests(n=nreq, rate_per_s=rate)
    for r in reqs:  # exchange tables depend only on the ladder: build them before the clock
        eng.estimate_bytes(r.problem)
    srv = Server(eng, budget_bytes=80 * 10 ** 9, slice_sweeps=100)
    srv.run(reqs)
    out = srv.summary()
    out.update({"rate_per_s": rate, "service_peak_attempts_per_s": peak})
    return out
