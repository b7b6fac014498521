"""Serving loop for many independent BCMG solves (continuous batching).

Requests (a Poisson problem of any size and geometry) arrive over time.  A
request is admitted as soon as its estimated device footprint
(bcmg_footprint_estimate) fits in the memory budget next to the requests
already on the GPU and a worker is free; it then builds its hierarchy on its
own library stream, evaluates its boundary data at the projection points,
and solves with the device-driven solve graph.  Requests in flight overlap on
the device (one stream each); a finished request frees its hierarchy and its
budget at once, so waiting requests are admitted while others still run.
Every solve is independent of the others, so its result is the same alone
and in the mix (the kernels are deterministic).

Latency of a request = completion time - arrival time (host clock).
"""

from __future__ import annotations

import heapq
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

from . import bcmg


@dataclass
class Request:
    """One solve.  phi, f: host float64 arrays with (N+1)^dim entries;
    g: callable mapping the (n_ghost, dim) CUDA tensor of projection points
    to the boundary values there; precision: bcmg.PREC_FP64 or PREC_MIXED."""
    rid: int
    dim: int
    N: int
    phi: np.ndarray
    f: np.ndarray
    g: Callable
    precision: int = bcmg.PREC_FP64
    rtol: float = 1e-10
    max_cycles: int = 100
    arrival: float = 0.0  # seconds after the start of the run
    keep_u: bool = False


@dataclass
class Result:
    rid: int
    cycles: int
    rel: float
    status: int
    arrival: float
    start: float
    done: float
    footprint: int
    u: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def solve_one(req: Request):
    """Build, solve and free one request on the current CUDA device;
    returns (cycles, rel, status, footprint, u or None)."""
    import torch
    phi = torch.from_numpy(np.ascontiguousarray(req.phi, dtype=np.float64)).cuda()
    f = torch.from_numpy(np.ascontiguousarray(req.f, dtype=np.float64)).cuda()
    s = bcmg.Solver(req.dim, req.N, phi, f, precision=req.precision)
    try:
        Q = s.ghost_points()
        s.set_boundary_values(req.g(Q).contiguous())
        u = torch.zeros_like(phi)
        cyc, rel, st = bcmg.solve_batch([s], [u], req.rtol, req.max_cycles)
        fp = s.memory_footprint()
        out = u.cpu().numpy() if req.keep_u else None
        return cyc[0], rel[0], st[0], fp, out
    finally:
        s.close()


class Server:
    """Admits requests by estimated footprint and runs up to `workers` of
    them at once, each on its own stream."""

    def __init__(self, mem_budget: int, workers: int = 8):
        self.mem_budget = int(mem_budget)
        self.workers = int(workers)

    def run(self, requests: list[Request]) -> list[Result]:
        """Replay the requests at their arrival times; return their results
        in completion order."""
        import torch
        dev = torch.cuda.current_device()
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            est = bcmg.footprint_estimate(r.dim, r.N, precision=r.precision)
            if est > self.mem_budget:
                raise ValueError("request %d needs %d bytes, more than the budget" % (r.rid, est))
        lock = threading.Condition()
        state = {"in_use": 0, "busy": 0}
        results: list[Result] = []
        t0 = time.perf_counter()

        def work(req: Request, est: int, start: float):
            torch.cuda.set_device(dev)
            try:
                with torch.cuda.stream(torch.cuda.Stream()):  # its own caller stream
                    cyc, rel, st, fp, u = solve_one(req)
            except bcmg.BcmgError as e:
                cyc, rel, st, fp, u = 0, float("nan"), e.code, 0, None
            done = time.perf_counter() - t0
            with lock:
                results.append(Result(req.rid, cyc, rel, st, req.arrival, start, done, fp, u))
                state["in_use"] -= est
                state["busy"] -= 1
                lock.notify_all()

        queue: list = []  # arrived, not yet admitted: (arrival, rid, req, est)
        i = 0
        with ThreadPoolExecutor(self.workers) as ex:
            while i < len(pending) or queue:
                now = time.perf_counter() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    r = pending[i]
                    heapq.heappush(queue, (r.arrival, r.rid, r,
                                           bcmg.footprint_estimate(r.dim, r.N, precision=r.precision)))
                    i += 1
                with lock:
                    # first come, first served; the head waits for memory
                    while queue and state["busy"] < self.workers and \
                            state["in_use"] + queue[0][3] <= self.mem_budget:
                        _, _, r, est = heapq.heappop(queue)
                        state["in_use"] += est
                        state["busy"] += 1
                        ex.submit(work, r, est, time.perf_counter() - t0)
                    if i < len(pending):
                        wait = max(0.0, pending[i].arrival - (time.perf_counter() - t0))
                    else:
                        wait = None
                    if queue or i < len(pending):
                        lock.wait(timeout=wait if not queue else 0.05 if wait is None else min(wait, 0.05))
            ex.shutdown(wait=True)
        return results


def percentiles(values, ps=(50, 99)):
    v = np.sort(np.asarray(values, dtype=float))
    return {p: float(np.percentile(v, p)) for p in ps} if v.size else {p: float("nan") for p in ps}
