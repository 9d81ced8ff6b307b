"""Shot-serving loop: continuous batching of propagation requests on one GPU.

The paper parallelises over shots (source experiments) because each shot's
forward modelling and gradient are independent (Sec. 3.4).  ``ShotServer``
serves such shots as they arrive:

- ``slots`` worker threads each own a ``wp_ctx`` (its own CUDA stream and a
  caching device pool, so wavefields, coefficients and checkpoints stay resident
  from one request to the next instead of being reallocated);
- a scheduler admits queued requests in arrival order, first fit, whenever a slot
  is free and the request's device-memory estimate fits in the budget (idle
  slots' cached memory is trimmed on demand, and each running slot's context is
  capped at its request's estimate); requests that arrive while others run are
  admitted as slots and memory free up, and their work overlaps on the device;
- every request returns its result or its error status without disturbing the
  other slots (bad input, CFL violation, over-budget, cancellation).

The library calls release the GIL (ctypes), so slots run concurrently.  The
executor is pluggable so that the scheduling logic can be exercised on the CPU.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Any, Callable

import numpy as np

from . import wavprop as W


@dataclass
class ShotRequest:
    """One shot: 'forward' returns receiver data, 'gradient' returns (dJ/dm, J)
    for J = 1/2 ||d - d_obs||^2.  Arrays are host numpy arrays."""

    id: int
    kind: str
    grid: W.Grid
    m: np.ndarray
    eta: np.ndarray
    wavelet: np.ndarray
    src: np.ndarray
    rec: np.ndarray
    d_obs: np.ndarray | None = None
    snap_interval: int = 20
    arrival: float = 0.0          # seconds on the server clock
    est_bytes: int = 0
    # filled by the server
    status: str = "queued"        # queued | running | done | error | cancelled
    result: Any = None
    misfit: float | None = None
    error: str | None = None
    error_status: int | None = None
    t_admit: float | None = None
    t_done: float | None = None
    slot: int | None = None
    done_event: threading.Event = field(default_factory=threading.Event, repr=False)

    @property
    def latency(self) -> float | None:
        return None if self.t_done is None else self.t_done - self.arrival


def estimate_bytes(req: ShotRequest) -> int:
    mode = 1 if req.kind == "gradient" else 0
    return W.wp_estimate_bytes(req.grid, len(req.src), len(req.rec), mode, req.snap_interval)


class _NvtxRange:
    """NVTX range "serve.<kind>" around one request (torch's NVTX binding; a no-op
    without it)."""

    def __init__(self, name: str):
        self.name = name
        self.pushed = False

    def __enter__(self):
        try:
            import torch
            torch.cuda.nvtx.range_push(self.name)
            self.pushed = True
        except Exception:
            pass
        return self

    def __exit__(self, *exc):
        if self.pushed:
            import torch
            torch.cuda.nvtx.range_pop()


def run_request(ctx_handle: int, req: ShotRequest):
    """Execute one request through the C ABI on a context (host arrays)."""
    with _NvtxRange(f"serve.{req.kind}"):
        return _run_request(ctx_handle, req)


def _run_request(ctx_handle: int, req: ShotRequest):
    if req.kind == "forward":
        return W.wp_forward(ctx_handle, req.grid, req.m, req.eta, req.wavelet, req.src, req.rec), None
    if req.kind == "gradient":
        d_obs = req.d_obs if req.d_obs is not None else np.zeros((req.grid.nt, len(req.rec)), np.float32)
        g, J = W.wp_fwi_gradient(ctx_handle, req.grid, req.m, req.eta, req.wavelet, req.src, d_obs, req.rec,
                                 req.snap_interval)
        return g, J
    raise ValueError(f"unknown request kind {req.kind!r}")


class _GpuSlots:
    """One wp_ctx per slot."""

    def __init__(self, nslots: int, device: int):
        self.ctx = [W.Context(device) for _ in range(nslots)]

    def in_use(self, s: int) -> int:
        return W.wp_bytes_in_use(self.ctx[s].handle)

    def trim(self, s: int, keep: int = 0):
        W.wp_trim(self.ctx[s].handle, keep)

    def cap(self, s: int, nbytes: int):
        W.wp_set_budget(self.ctx[s].handle, nbytes)

    def run(self, s: int, req: ShotRequest):
        return run_request(self.ctx[s].handle, req)

    def close(self):
        for c in self.ctx:
            c.close()


class ShotServer:
    """Continuous-batching server of ShotRequests (see module docstring)."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int | None = None, device: int = 0,
                 backend=None, clock: Callable[[], float] = time.perf_counter):
        self.nslots = slots
        self.backend = backend if backend is not None else _GpuSlots(slots, device)
        if hbm_budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget_bytes = int(0.85 * free)
        self.budget = int(hbm_budget_bytes)
        self.clock = clock
        self.t0 = clock()
        self.cv = threading.Condition()
        self.queue: deque[ShotRequest] = deque()
        self.free_slots = list(range(slots))
        self.slot_reserved = [0] * slots   # bytes reserved by the running request of each slot
        self.peak_reserved = 0
        self.closed = False
        self.completed: list[ShotRequest] = []
        self.work: list[ShotRequest | None] = [None] * slots
        self.threads = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(slots)]
        for t in self.threads:
            t.start()
        self.sched = threading.Thread(target=self._scheduler, daemon=True)
        self.sched.start()

    # -- client side -------------------------------------------------------
    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: ShotRequest) -> ShotRequest:
        if not req.est_bytes:
            req.est_bytes = estimate_bytes(req)
        with self.cv:
            if req.arrival == 0.0:
                req.arrival = self.now()
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def cancel(self, req: ShotRequest) -> bool:
        """Cancel a request that has not started; True if it was cancelled."""
        with self.cv:
            if req.status == "queued" and req in self.queue:
                self.queue.remove(req)
                self._finish(req, "cancelled")
                return True
        return False

    def drain(self, timeout: float | None = None) -> bool:
        with self.cv:
            return self.cv.wait_for(lambda: not self.queue and len(self.free_slots) == self.nslots, timeout)

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        self.sched.join()
        if hasattr(self.backend, "close"):
            self.backend.close()

    # -- scheduling ----------------------------------------------------------
    def _idle_cached(self) -> int:
        return sum(self.backend.in_use(s) for s in self.free_slots)

    def _reserved(self) -> int:
        return sum(self.slot_reserved)

    def _try_admit(self) -> bool:
        """Admit the first queued request that fits (caller holds the lock)."""
        if not self.free_slots or not self.queue:
            return False
        for req in list(self.queue):
            need = int(req.est_bytes * 1.05) + (64 << 20)
            if need > self.budget:
                self.queue.remove(req)
                req.error_status = W.WP_ENOMEM
                self._finish(req, "error", f"needs ~{need} bytes, more than the server budget {self.budget}")
                return True
            if self._reserved() + need > self.budget:
                continue
            # pick the idle slot whose resident pool is largest (most reuse), then
            # trim idle pools until the reservation fits beside everything resident
            slot = max(self.free_slots, key=lambda s: self.backend.in_use(s))
            others = [s for s in self.free_slots if s != slot]
            if self._reserved() + need + sum(self.backend.in_use(s) for s in others) + \
                    max(0, self.backend.in_use(slot) - need) > self.budget:
                for s in sorted(others, key=lambda s: -self.backend.in_use(s)):
                    self.backend.trim(s, 0)
                    if self._reserved() + need + sum(self.backend.in_use(o) for o in others) <= self.budget:
                        break
            if self.backend.in_use(slot) > need:
                self.backend.trim(slot, need)
            self.queue.remove(req)
            self.free_slots.remove(slot)
            self.slot_reserved[slot] = need
            self.peak_reserved = max(self.peak_reserved, self._reserved())
            self.backend.cap(slot, need)
            req.status = "running"
            req.slot = slot
            req.t_admit = self.now()
            self.work[slot] = req
            self.cv.notify_all()
            return True
        return False

    def _scheduler(self):
        with self.cv:
            while not self.closed:
                if not self._try_admit():
                    self.cv.wait(0.05)

    def _finish(self, req: ShotRequest, status: str, error: str | None = None):
        req.status = status
        req.error = error
        req.t_done = self.now()
        self.completed.append(req)
        req.done_event.set()
        self.cv.notify_all()

    def _worker(self, s: int):
        while True:
            with self.cv:
                self.cv.wait_for(lambda: self.work[s] is not None or self.closed)
                if self.work[s] is None:
                    return
                req = self.work[s]
            status, err = "done", None
            try:
                req.result, req.misfit = self.backend.run(s, req)
            except W.WpError as e:
                status, err = "error", str(e)
                req.error_status = e.status
            except Exception as e:  # noqa: BLE001 - a request never takes the server down
                status, err = "error", repr(e)
            with self.cv:
                self.work[s] = None
                self.slot_reserved[s] = 0
                self.free_slots.append(s)
                self._finish(req, status, err)


# ---------------------------------------------------------------------------
# load generation and the two ways of serving a stream
# ---------------------------------------------------------------------------

def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of `rate` requests per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def serve_stream(requests: list[ShotRequest], arrivals, slots: int = 4, hbm_budget_bytes: int | None = None,
                 device: int = 0) -> dict:
    """Submit each request at its arrival time to a ShotServer; wait for all."""
    server = ShotServer(slots=slots, hbm_budget_bytes=hbm_budget_bytes, device=device)
    try:
        for req, t in zip(requests, arrivals):
            req.est_bytes = estimate_bytes(req)
            delay = t - server.now()
            if delay > 0:
                time.sleep(delay)
            req.arrival = float(t)
            server.submit(req)
        server.drain()
        makespan = server.now()
        peak = server.peak_reserved
    finally:
        server.close()
    return summarize(requests, makespan, extra={"slots": slots, "peak_reserved_bytes": peak,
                                                "budget_bytes": server.budget})


def serve_sequential_plain(requests: list[ShotRequest], arrivals, device: int = 0,
                           reuse_context: bool = False) -> dict:
    """The same stream served one request at a time, in arrival order, with no
    overlap.  By default each request gets a fresh context (nothing resident
    between requests: the plain one-call-per-shot baseline); with reuse_context
    one context serves them all, so its device pool and kernels stay warm and the
    only thing missing against the server is the overlap of requests."""
    t0 = time.perf_counter()
    shared = W.Context(device) if reuse_context else None
    try:
        for req, t in zip(requests, arrivals):
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            req.arrival = float(t)
            req.t_admit = time.perf_counter() - t0
            try:
                if shared is not None:
                    req.result, req.misfit = run_request(shared.handle, req)
                else:
                    with W.Context(device) as c:
                        req.result, req.misfit = run_request(c.handle, req)
                req.status = "done"
            except W.WpError as e:
                req.status, req.error, req.error_status = "error", str(e), e.status
            req.t_done = time.perf_counter() - t0
    finally:
        if shared is not None:
            shared.close()
    makespan = time.perf_counter() - t0
    return summarize(requests, makespan, extra={"slots": 1, "context": "reused" if reuse_context else "fresh"})


def summarize(requests: list[ShotRequest], makespan: float, extra: dict | None = None) -> dict:
    lat = np.array([r.latency for r in requests if r.status == "done"])
    ok = len(lat)
    out = {
        "requests": len(requests), "completed": ok,
        "errors": sum(1 for r in requests if r.status == "error"),
        "makespan_s": makespan,
        "shots_per_hour": 3600.0 * ok / makespan if makespan > 0 else 0.0,
        "p50_latency_s": float(np.percentile(lat, 50)) if ok else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if ok else None,
        "mean_latency_s": float(lat.mean()) if ok else None,
    }
    errs = [f"{r.id}:{r.kind}: {r.error}" for r in requests if r.status == "error"]
    if errs:
        out["error_messages"] = errs[:5]
    if extra:
        out.update(extra)
    return out


def make_request(spec: dict, ident: int | None = None) -> ShotRequest:
    """Build a ShotRequest (host arrays) from a serving-stream spec of synth."""
    from . import synth
    model = synth.request_model(spec)
    k = model.space_order
    dt = 0.9 * W.wp_cfl_dt(W.Grid(model.shape, model.spacing, model.origin, k), model.vmax)
    grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, int(spec["nt"]))
    d_obs = np.zeros((grid.nt, len(model.rec)), np.float32) if spec["kind"] == "gradient" else None
    return ShotRequest(id=spec["id"] if ident is None else ident, kind=spec["kind"], grid=grid, m=model.m32(),
                       eta=model.eta32(), wavelet=model.wavelet(dt, grid.nt), src=model.src, rec=model.rec,
                       d_obs=d_obs, snap_interval=20)
