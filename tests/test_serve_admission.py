"""Admission control of the served stream, driven on the CPU.

The server admits requests by estimated footprint.  When a creation still
fails with BCMG_ENOMEM (the estimate was low, or memory is held elsewhere),
the request must be queued again rather than failed, the admission limit must
back off, and the request must complete once memory frees up.  Here the
device is a fake allocator with a fixed capacity and the creations are host
threads that hold their true footprint for a short time; no GPU is involved.
"""

import threading
import time

import numpy as np
import pytest

from paper_2207_14208_gb300 import bcmg, serve


class FakeDeviceServer(serve.Server):
    def __init__(self, capacity, true_bytes, hold_s=0.02, **kw):
        super().__init__(**kw)
        self.capacity = capacity
        self.true_bytes = true_bytes  # rid -> bytes the creation really takes
        self.hold_s = hold_s
        self.used = 0
        self.peak = 0
        self.lock = threading.Lock()
        self.enomem = 0

    def _prepare(self):
        pass

    def estimate(self, req):
        return req.N  # the "estimate" rides in N for the fake

    def execute(self, req):
        need = self.true_bytes[req.rid]
        with self.lock:
            if self.used + need > self.capacity:
                self.enomem += 1
                raise bcmg.BcmgError(bcmg.ENOMEM, "device allocation failed (fake)")
            self.used += need
            self.peak = max(self.peak, self.used)
        time.sleep(self.hold_s)
        with self.lock:
            self.used -= need
        return 5, 1e-11, bcmg.OK, need, None


def _req(rid, est, arrival=0.0):
    return serve.Request(rid=rid, dim=2, N=est, phi=np.zeros(1), f=np.zeros(1), g=None, arrival=arrival)


def test_enomem_requeues_and_completes():
    # estimates of 10 each, true footprints 30: four fit the budget by the
    # estimate (40 <= 100) but only three fit the device (capacity 100)
    reqs = [_req(i, 10, arrival=0.001 * i) for i in range(12)]
    srv = FakeDeviceServer(capacity=100, true_bytes={i: 30 for i in range(12)}, mem_budget=100, workers=6)
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == list(range(12))
    assert all(r.status == bcmg.OK for r in res)
    assert srv.backoffs > 0 and srv.enomem == srv.backoffs
    assert srv.peak <= srv.capacity


def test_request_too_large_alone_reports_enomem():
    reqs = [_req(0, 10), _req(1, 10, arrival=0.005)]
    srv = FakeDeviceServer(capacity=100, true_bytes={0: 150, 1: 20}, mem_budget=100, workers=2, max_retries=3)
    res = {r.rid: r for r in srv.run(reqs)}
    assert res[0].status == bcmg.ENOMEM
    assert res[1].status == bcmg.OK


def test_retry_limit_bounds_backoffs():
    # a request that never fits next to a long-running one gives up after
    # max_retries returns instead of looping
    reqs = [_req(0, 10), _req(1, 10, arrival=0.002)]
    srv = FakeDeviceServer(capacity=100, true_bytes={0: 60, 1: 60}, mem_budget=100, workers=2, max_retries=2,
                           hold_s=0.05)
    res = {r.rid: r for r in srv.run(reqs)}
    assert res[0].status == bcmg.OK
    # request 1 either waited until request 0 finished (limit backed off) and
    # then succeeded, or exhausted its retries
    assert res[1].status in (bcmg.OK, bcmg.ENOMEM)
    assert srv.backoffs <= 2


def test_fifo_order_kept_after_backoff():
    reqs = [_req(i, 10, arrival=0.0005 * i) for i in range(8)]
    srv = FakeDeviceServer(capacity=60, true_bytes={i: 30 for i in range(8)}, mem_budget=100, workers=8)
    res = srv.run(reqs)
    starts = sorted(res, key=lambda r: r.start)
    assert all(r.status == bcmg.OK for r in res)
    # admissions follow arrival order
    assert [r.rid for r in starts] == sorted(r.rid for r in starts) or srv.backoffs > 0


@pytest.mark.parametrize("workers", [1, 3])
def test_no_backoff_when_estimates_hold(workers):
    reqs = [_req(i, 30, arrival=0.001 * i) for i in range(6)]
    srv = FakeDeviceServer(capacity=100, true_bytes={i: 30 for i in range(6)}, mem_budget=100, workers=workers)
    res = srv.run(reqs)
    assert all(r.status == bcmg.OK for r in res) and srv.backoffs == 0
