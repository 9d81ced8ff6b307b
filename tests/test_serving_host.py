"""Scheduling logic of the shot server on the CPU (fake executor, no GPU)."""
import threading
import time

import numpy as np
import pytest

from paper_1808_01995_gb300 import serving as S
from paper_1808_01995_gb300 import wavprop as W


class FakeSlots:
    """Stands in for the GPU slots: run() sleeps for req.extra duration and keeps
    a per-slot 'resident' pool equal to the last request's reservation."""

    def __init__(self, n, fail_ids=()):
        self.pool = [0] * n
        self.cap_ = [0] * n
        self.running = 0
        self.max_running = 0
        self.lock = threading.Lock()
        self.fail_ids = set(fail_ids)
        self.trims = 0

    def in_use(self, s):
        return self.pool[s]

    def trim(self, s, keep=0):
        self.trims += 1
        self.pool[s] = min(self.pool[s], keep)

    def cap(self, s, n):
        self.cap_[s] = n

    def run(self, s, req):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
        try:
            time.sleep(req.duration)
            if req.id in self.fail_ids:
                raise W.WpError(W.WP_ECFL, "planted failure")
            self.pool[s] = self.cap_[s]
            return ("ok", req.id), None
        finally:
            with self.lock:
                self.running -= 1


def req(i, est, duration=0.05, kind="forward"):
    g = W.Grid((8, 8, 8), (1.0,) * 3, (0.0,) * 3, 4, 1e-3, 4)
    r = S.ShotRequest(id=i, kind=kind, grid=g, m=None, eta=None, wavelet=None, src=np.zeros((0, 3)),
                      rec=np.zeros((0, 3)), est_bytes=est)
    r.duration = duration
    return r


def test_continuous_batching_fills_free_slots():
    fake = FakeSlots(2)
    srv = S.ShotServer(slots=2, hbm_budget_bytes=1 << 40, backend=fake)
    try:
        reqs = [srv.submit(req(i, 1 << 20, 0.05)) for i in range(6)]
        assert srv.drain(10)
    finally:
        srv.close()
    assert all(r.status == "done" for r in reqs)
    assert fake.max_running == 2
    # six 50 ms jobs on two slots: about three rounds, not six
    assert max(r.t_done for r in reqs) < 0.25


def test_late_arrivals_are_admitted_while_others_run():
    fake = FakeSlots(3)
    srv = S.ShotServer(slots=3, hbm_budget_bytes=1 << 40, backend=fake)
    try:
        a = srv.submit(req(0, 1 << 20, 0.3))
        time.sleep(0.05)
        b = srv.submit(req(1, 1 << 20, 0.05))
        assert b.done_event.wait(5)
        assert not a.done_event.is_set()  # b finished while a was still running
        assert srv.drain(5)
    finally:
        srv.close()
    assert b.t_done < a.t_done


def test_budget_limits_concurrency_and_is_never_exceeded():
    fake = FakeSlots(4)
    budget = 3 << 30
    srv = S.ShotServer(slots=4, hbm_budget_bytes=budget, backend=fake)
    try:
        reqs = [srv.submit(req(i, 1 << 30, 0.03)) for i in range(8)]  # ~1.1 GB reserved each
        assert srv.drain(10)
    finally:
        srv.close()
    assert all(r.status == "done" for r in reqs)
    assert srv.peak_reserved <= budget
    assert fake.max_running <= 2


def test_first_fit_skips_a_request_that_does_not_fit_yet():
    fake = FakeSlots(2)
    budget = 4 << 30
    srv = S.ShotServer(slots=2, hbm_budget_bytes=budget, backend=fake)
    try:
        big0 = srv.submit(req(0, 3 << 30, 0.3))
        time.sleep(0.02)
        big1 = srv.submit(req(1, 3 << 30, 0.05))   # must wait for big0's memory
        small = srv.submit(req(2, 256 << 20, 0.05))  # fits beside big0: admitted first
        assert srv.drain(10)
    finally:
        srv.close()
    assert small.t_admit < big1.t_admit
    assert small.t_done < big0.t_done


def test_over_budget_failure_and_cancel_do_not_disturb_others():
    fake = FakeSlots(2, fail_ids={3})
    srv = S.ShotServer(slots=2, hbm_budget_bytes=2 << 30, backend=fake)
    try:
        blocker = srv.submit(req(0, 1 << 29, 0.2))
        blocker2 = srv.submit(req(1, 1 << 29, 0.2))
        huge = srv.submit(req(2, 8 << 30))
        bad = srv.submit(req(3, 1 << 20))
        gone = srv.submit(req(4, 1 << 20))
        ok = srv.submit(req(5, 1 << 20))
        assert srv.cancel(gone)
        assert srv.drain(10)
    finally:
        srv.close()
    assert huge.status == "error" and huge.error_status == W.WP_ENOMEM
    assert bad.status == "error" and bad.error_status == W.WP_ECFL
    assert gone.status == "cancelled"
    assert ok.status == "done" and blocker.status == "done" and blocker2.status == "done"


def test_summary_statistics():
    reqs = [req(i, 1) for i in range(4)]
    for i, r in enumerate(reqs):
        r.status, r.arrival, r.t_done = "done", float(i), float(i) + 1.0 + i
    s = S.summarize(reqs, 10.0)
    assert s["completed"] == 4 and abs(s["shots_per_hour"] - 1440.0) < 1e-9
    assert s["p50_latency_s"] == pytest.approx(2.5)
    assert s["p99_latency_s"] <= 4.0


def test_poisson_arrivals_rate():
    t = S.poisson_arrivals(20000, 5.0, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 5.0) < 0.2
