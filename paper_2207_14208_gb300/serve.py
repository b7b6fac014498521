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


class _PinnedPool:
    """Page-locked host staging buffers for the requests' phi and f, kept for
    the life of the process (freeing page-locked memory waits for the whole
    device).  Sizes are rounded up to powers of two so that buffers are
    reused across request sizes; at most two per request in flight exist
    per size class."""

    def __init__(self):
        self._free: list = []
        self._lock = threading.Lock()

    def get(self, n: int):
        import torch
        cap = 1 << max(17, (int(n) - 1).bit_length())  # doubles
        with self._lock:
            for i, b in enumerate(self._free):
                if b.numel() == cap:
                    return self._free.pop(i)
        return torch.empty(cap, dtype=torch.float64, pin_memory=True)

    def put(self, b) -> None:
        with self._lock:
            self._free.append(b)


_pinned = _PinnedPool()


def solve_one(req: Request):
    """Build, solve and free one request on the current CUDA device;
    returns (cycles, rel, status, footprint, u or None).  phi and f go
    through page-locked staging buffers (pageable copies from many threads
    serialise in the driver); creation needs phi only, so f is copied on a
    second stream while the hierarchy is built and set afterwards."""
    import torch
    n = req.phi.size
    main = torch.cuda.current_stream()
    side = _side_stream()
    bp, bf = _pinned.get(n), _pinned.get(n)
    try:
        np.copyto(bp[:n].numpy(), np.asarray(req.phi, dtype=np.float64).reshape(-1))
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        phi.copy_(bp[:n], non_blocking=True)
        np.copyto(bf[:n].numpy(), np.asarray(req.f, dtype=np.float64).reshape(-1))
        side.wait_stream(main)
        with torch.cuda.stream(side):
            f = torch.empty(n, dtype=torch.float64, device="cuda")
            f.copy_(bf[:n], non_blocking=True)
        s = bcmg.Solver(req.dim, req.N, phi, None, precision=req.precision)
        main.wait_stream(side)
        f.record_stream(main)
        s.set_rhs(f)
    except BaseException:
        main.synchronize()  # streams, not the device: another thread may be capturing
        side.synchronize()
        _pinned.put(bp)
        _pinned.put(bf)
        raise
    try:
        # the staging buffers are free once the copies are done
        main.synchronize()
        _pinned.put(bp)
        _pinned.put(bf)
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
    them at once, each on its own stream.

    If a creation still runs out of device memory (BCMG_ENOMEM: the estimate
    was low for that geometry, or other users hold memory), the request is
    not failed: its budget is released, the admission limit backs off to the
    memory the other requests in flight hold, and the request goes back to
    the head of the queue (its arrival order is kept) to be admitted again
    once enough of them have finished.  After `max_retries` such returns, or
    if it fails with nothing else in flight, its result carries the ENOMEM
    status.  The limit returns to `mem_budget` after the next success."""

    def __init__(self, mem_budget: int, workers: int = 8, max_retries: int = 8):
        self.mem_budget = int(mem_budget)
        self.workers = int(workers)
        self.max_retries = int(max_retries)
        self.backoffs = 0  # ENOMEM returns of the last run

    # device-facing parts (a test replaces them to drive the admission logic
    # without a GPU)
    def estimate(self, req: Request) -> int:
        return bcmg.footprint_estimate(req.dim, req.N, precision=req.precision)

    def execute(self, req: Request):
        """(cycles, rel, status, footprint, u) of one request; raises
        bcmg.BcmgError on a failed creation."""
        import torch
        torch.cuda.set_device(self._dev)
        with torch.cuda.stream(torch.cuda.Stream()):  # its own caller stream
            return solve_one(req)

    def _prepare(self):
        import torch
        self._dev = torch.cuda.current_device()

    def run(self, requests: list[Request]) -> list[Result]:
        """Replay the requests at their arrival times; return their results
        in completion order."""
        self._prepare()
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            est = self.estimate(r)
            if est > self.mem_budget:
                raise ValueError("request %d needs %d bytes, more than the budget" % (r.rid, est))
        lock = threading.Condition()
        state = {"in_use": 0, "busy": 0, "limit": self.mem_budget}
        retries: dict = {}
        results: list[Result] = []
        queue: list = []  # arrived, not yet admitted: (arrival, rid, req, est)
        self.backoffs = 0
        t0 = time.perf_counter()

        def work(req: Request, est: int, start: float):
            try:
                cyc, rel, st, fp, u = self.execute(req)
            except bcmg.BcmgError as e:
                with lock:
                    others = state["in_use"] - est
                    if e.code == bcmg.ENOMEM and others > 0 and retries.get(req.rid, 0) < self.max_retries:
                        # back off: admit no more than what the others hold
                        # until one of them finishes, and queue it again
                        retries[req.rid] = retries.get(req.rid, 0) + 1
                        self.backoffs += 1
                        state["in_use"] -= est
                        state["busy"] -= 1
                        state["limit"] = max(others, est)
                        heapq.heappush(queue, (req.arrival, req.rid, req, est))
                        lock.notify_all()
                        return
                cyc, rel, st, fp, u = 0, float("nan"), e.code, 0, None
            done = time.perf_counter() - t0
            with lock:
                results.append(Result(req.rid, cyc, rel, st, req.arrival, start, done, fp, u))
                state["in_use"] -= est
                state["busy"] -= 1
                if st != bcmg.ENOMEM:
                    state["limit"] = self.mem_budget
                lock.notify_all()

        i = 0
        with ThreadPoolExecutor(self.workers) as ex:
            while True:
                with lock:
                    if i >= len(pending) and not queue and state["busy"] == 0:
                        break
                now = time.perf_counter() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    r = pending[i]
                    est = self.estimate(r)
                    with lock:
                        heapq.heappush(queue, (r.arrival, r.rid, r, est))
                    i += 1
                with lock:
                    # first come, first served; the head waits for memory
                    while queue and state["busy"] < self.workers and \
                            (state["in_use"] + queue[0][3] <= state["limit"] or state["busy"] == 0):
                        _, _, r, est = heapq.heappop(queue)
                        state["in_use"] += est
                        state["busy"] += 1
                        ex.submit(work, r, est, time.perf_counter() - t0)
                    if i < len(pending):
                        wait = max(0.0, pending[i].arrival - (time.perf_counter() - t0))
                    else:
                        wait = None
                    lock.wait(timeout=0.05 if wait is None else min(wait, 0.05))
            ex.shutdown(wait=True)
        return results


_tls = threading.local()


def _side_stream():
    """This thread's second stream (the f copy during creation)."""
    import torch
    st = getattr(_tls, "side", None)
    if st is None:
        st = _tls.side = torch.cuda.Stream()
    return st


def percentiles(values, ps=(50, 99)):
    v = np.sort(np.asarray(values, dtype=float))
    return {p: float(np.percentile(v, p)) for p in ps} if v.size else {p: float("nan") for p in ps}
