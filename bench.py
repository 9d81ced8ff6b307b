#!/usr/bin/env python
"""Throughput benchmark of the GB300 damped-acoustic propagator.

One step = one forward shot of the 3D stencil sweep workload: 256^3 interior at
10 m plus a 40-point damping layer (336^3 grid), 8 flat layers 1.5 -> 4.5 km/s,
space order 8, dt = 0.9 x CFL, 1000 time steps, one 15 Hz Ricker source and
128 x 128 off-grid receivers (coefficient setup, stencil, injection,
interpolation and the time loop all run in the CUDA library).

value  = grid points updated per second over all ranks (Gpts/s), inputs resident
         in HBM, device-timed with CUDA events.
e2e    = same metric through the host-array C-ABI call (m, eta, wavelet copied in
         from pinned host memory and the receiver data copied out every step).
roofline: the stencil kernel's compulsory bytes per launch over its live average
         duration (CUDA events on the library's stream), against the measured
         HBM copy bandwidth.
cpu_baseline / --impl reference: the FP64 CPU oracle on a bounded sample.
Further single-GPU legs: the FWI gradient (280^3), shot serving, the 592x592x480
SO16 workload, the CFD examples and paper_context (the paper's time-to-solution
experiment: 1000 ms of modelling at SO16 on a 512^3 grid, quoted beside the
paper's CPU figure as context only).

Multi-GPU (torchrun): replicas only (one independent shot per GPU, no collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s & %HBM roofline, SO8 3D acoustic; shots/h + p99 served vs plain"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--space-order", type=int, default=8)
    p.add_argument("--nt", type=int, default=1000)
    p.add_argument("--n", type=int, default=256, help="interior points per axis")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--serving", type=int, default=256,
                   help="requests of the shot-serving stream (0 skips the serving leg)")
    p.add_argument("--serving-calibration", type=int, default=24,
                   help="requests timed one by one to set the arrival rate (1.25x their service rate)")
    p.add_argument("--serving-capacity", action="store_true",
                   help="also serve the whole stream queued at t = 0 (served and plain)")
    p.add_argument("--serving-slots", type=int, default=4)
    p.add_argument("--serving-scale", type=float, default=1.0,
                   help="scale of the request sizes and nt (1.0 = 128..320 x 128..320 x 128..200 + 40, nt 500..2000)")
    p.add_argument("--gradient", type=int, default=3,
                   help="timed FWI gradients of the 200^3 + 40 blobs workload (0 skips the gradient leg)")
    p.add_argument("--gradient-nt", type=int, default=1500,
                   help="time steps of the gradient workload (1500; fewer only for profiling)")
    p.add_argument("--cfd-n", type=int, default=8192,
                   help="edge of the 2D CFD example fields (0 skips the CFD leg)")
    p.add_argument("--large-nt", type=int, default=3000,
                   help="time steps of the full-size SO16 salt leg (0 skips it)")
    p.add_argument("--context", type=lambda v: [int(x) for x in v.split(",") if x.strip() and int(x) > 0],
                   default=[512], help="grid edges of the paper-context leg (SO16, 1000 ms of modelling); "
                   "'0' skips it")
    p.add_argument("--checkpoints", type=int, default=20,
                   help="stored states of the binomial-checkpointing gradient timed beside it (0 skips it)")
    p.add_argument("--no-full-history", dest="full_history", action="store_false",
                   help="skip the full-history gradient (snap_interval 1, ~135 GB) timed beside the snapshot one")
    p.add_argument("--no-reconstruct", dest="reconstruct", action="store_false",
                   help="skip the boundary-reconstruction gradient timed beside the snapshot one")
    p.add_argument("--orders", type=lambda v: [int(x) for x in v.split(",") if x.strip() and int(x) > 0],
                   default=[4, 8, 12, 16], help="space orders of the roofline sweep ('0' skips it)")
    p.add_argument("--order-shots", type=int, default=3, help="timed shots per order of the roofline sweep")
    p.add_argument("--profile-every", type=int, default=10,
                   help="bracket every N-th stencil launch with CUDA events in the timed region")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_init(backend: str | None = None):
    """(world, rank, local_rank) from the torchrun environment; initialises the
    process group for N > 1 (NCCL on GPUs, gloo otherwise)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend or ("nccl" if torch.cuda.is_available() else "gloo"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Maximum of a scalar over all ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, points_per_rank, seconds_max):
    """Replicas: every rank updates the same number of points; the job's rate is
    all ranks' points over the slowest rank's time (Gpts/s)."""
    return world * points_per_rank / seconds_max / 1e9


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload(args):
    from paper_1808_01995_gb300 import synth
    model = synth.layers_3d(space_order=args.space_order, n=args.n, nt=args.nt)
    return model


def describe(model, nt, dt):
    n = model.shape
    return {"workload": f"layers3d {model.shape[0] - 2 * model.nbl}^3 + {model.nbl}-pt layer ({n[0]}x{n[1]}x{n[2]}) "
                        f"SO{model.space_order} forward, nt={nt}, 1 Ricker source, {len(model.rec)} receivers",
            "grid": list(n), "space_order": model.space_order, "nt": nt, "dt_s": dt,
            "l2": "inputs larger than L2 (four 4-byte fields of the grid per step)",
            "parallelism": "replicas (one shot per GPU)"}


def algorithmic_bytes_per_launch(model):
    """Compulsory stencil bytes of one time step: read u^n, u^{n-1}, b, write u^{n+1}
    (16 B per point) plus s (4 B) where eta != 0."""
    npts = int(np.prod(model.shape))
    ndamp = int(np.count_nonzero(model.eta))
    return 16 * npts + 4 * ndamp, npts, ndamp


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(space_order, grid):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"stencil3d_fwd_so{space_order}_{grid}.md")
    if not os.path.exists(path):
        return None
    name = "stencil3d.cuh" if space_order <= 8 else "stencil3d_hi.cuh"
    src = open(os.path.join(ROOT, "paper_1808_01995_gb300", "csrc", name), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ": " in line and line.startswith("- "):
            k, v = line[2:].split(": ", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get(f"{name} sha256[:16]") != sha:
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# oracle legs (CPU)
# ---------------------------------------------------------------------------
def oracle_timed(model, dt, steps):
    """Seconds of one FP64 oracle forward of `steps` time steps on the full grid
    (the call allocates and zeroes its FP64 fields first)."""
    import oracle as O
    g = O.Grid(model.shape, model.spacing, model.origin, model.space_order, dt, steps)
    q = model.wavelet(dt, steps)
    m, eta = model.m32(), model.eta32()
    t0 = time.perf_counter()
    O.forward(g, m, eta, q, model.src, model.rec)
    return time.perf_counter() - t0


def oracle_sample(model, dt, budget_s):
    """The FP64 oracle's forward rate on the full grid over a bounded number of time
    steps: the steps are grown until one run takes about budget_s / 2, and the rate
    is taken from the difference with a one-step run, so that the per-call setup
    (allocating and zeroing the FP64 fields) cancels.
    Returns (Gpts/s, steps, seconds of the longest run, threads)."""
    import oracle as O
    nthreads = O.num_threads()
    t1 = oracle_timed(model, dt, 1)
    steps = 2
    while True:
        el = oracle_timed(model, dt, steps)
        if el >= 0.5 * budget_s or steps >= 4096:
            break
        steps = max(steps + 1, min(steps * 8, int(steps * 0.6 * budget_s / max(el - t1, 1e-3))))
    return np.prod(model.shape) * (steps - 1) / max(el - t1, 1e-9) / 1e9, steps, el, nthreads


def oracle_sample_one_thread(model, dt, nthreads, budget_s=2.0):
    """The oracle's forward rate on one host thread (a short sample), then the
    thread count restored."""
    import oracle as O
    O.set_threads(1)
    try:
        rate, steps, el, _ = oracle_sample(model, dt, budget_s)
    finally:
        O.set_threads(nthreads)
    return rate, steps, el


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores.  One bench step is a
    bounded sample of the shot (n of its time steps, n fixed in the warm-up so the
    whole run stays within about --cpu-seconds); ms_per_step is the time of that
    sample as run, and the rate (value) is taken from the difference with a
    one-step run, so that the oracle's per-call setup cancels."""
    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    from paper_1808_01995_gb300 import synth  # noqa: F401  (inputs only)
    import oracle as O
    t_start = time.perf_counter()
    model = workload(args)
    dt = 0.9 * O.cfl_dt(model.spacing, args.space_order, model.vmax)
    nthreads = O.num_threads()
    npts = int(np.prod(model.shape))
    # warm-up: the one-step time (setup + 1 step) and the sample length
    t1 = min(oracle_timed(model, dt, 1) for _ in range(max(args.warmup, 1)))
    per_step_s = max(0.5, args.cpu_seconds / max(args.steps, 1))
    t_probe = oracle_timed(model, dt, 4)
    step_s = max((t_probe - t1) / 3, 1e-4)
    n = int(max(2, min(args.nt, 1 + (per_step_s - t1) / step_s)))
    times = [oracle_timed(model, dt, n) for _ in range(args.steps)]
    t_med = float(np.median(times))
    v = npts * (n - 1) / max(t_med - t1, 1e-9) / 1e9
    timed_s = float(sum(times))
    sample = (f"FP64 oracle forward on the full {model.shape} grid, {n} of the shot's {args.nt} time steps "
              f"per bench step; rate from the difference with a one-step run ({t1:.2f} s, the setup)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_med * 1e3, "ms_per_step_is": f"one bench step = {n} oracle time steps, as run",
            "ms_per_shot_extrapolated": npts * args.nt / (v * 1e9) * 1e3,
            "seconds_timed": timed_s, "seconds_total": time.perf_counter() - t_start,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(model, args.nt, dt),
            "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": nthreads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def serving_leg(args):
    """Shot-serving stream (the 256-request Poisson stream by default): arrivals at
    1.25x the plain sequential service rate (estimated on the first requests), served by
    ShotServer (continuous batching) and, for comparison, one request at a time
    with a fresh context each (plain calls) and one request at a time on one
    reused context (no overlap, but nothing re-created: what the server gains
    beyond that is the overlap)."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1808_01995_gb300 import serving as S
    from paper_1808_01995_gb300 import synth
    from paper_1808_01995_gb300 import wavprop as W
    specs = synth.serving_requests(count=args.serving, size_scale=args.serving_scale)
    with ThreadPoolExecutor(8) as ex:
        base = list(ex.map(S.make_request, specs))

    def fresh():
        out = []
        for r in base:
            c = S.ShotRequest(id=r.id, kind=r.kind, grid=r.grid, m=r.m, eta=r.eta, wavelet=r.wavelet, src=r.src,
                              rec=r.rec, d_obs=r.d_obs, snap_interval=r.snap_interval)
            out.append(c)
        return out

    # calibration: plain sequential service times (fresh context per request) of a
    # sample of the stream; also warms the host caches
    import time as _t
    ncal = min(len(base), args.serving_calibration)
    service = []
    for r in fresh()[:ncal]:
        t0 = _t.perf_counter()
        with W.Context(0) as c:
            S.run_request(c.handle, r)
        service.append(_t.perf_counter() - t0)
    # the sizes and nt of the stream vary about tenfold: fit the service time of the
    # sample as a per-kind cost per point-step and predict the whole stream's mean
    work = np.array([float(np.prod(r.grid.shape)) * r.grid.nt for r in base])
    grad = np.array([r.kind == "gradient" for r in base], dtype=float)
    A = np.stack([work[:ncal] * (1 - grad[:ncal]), work[:ncal] * grad[:ncal], np.ones(ncal)], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.array(service), rcond=None)
    pred = np.stack([work * (1 - grad), work * grad, np.ones(len(base))], axis=1) @ coef
    mean_service = float(np.mean(pred)) if np.all(pred > 0) else float(np.mean(service))
    mu = 1.0 / mean_service
    rate = 1.25 * mu
    arrivals = S.poisson_arrivals(len(base), rate, seed=1808 + 4)
    served = S.serve_stream(fresh(), arrivals, slots=args.serving_slots)
    plain = S.serve_sequential_plain(fresh(), arrivals)
    reused = S.serve_sequential_plain(fresh(), arrivals, reuse_context=True)
    kinds = [s["kind"] for s in specs]

    def ratio(a, b):
        return a / b if a and b else None

    out = {"requests": len(base), "forward": kinds.count("forward"), "gradient": kinds.count("gradient"),
           "arrival_rate_per_s": rate, "sequential_service_rate_per_s": mu,
           "mean_service_s": mean_service, "calibration_mean_service_s": float(np.mean(service)),
           "calibration_requests": ncal,
           "service_model": "t = a * points * nt (forward) or b * points * nt (gradient) + c, fitted on the "
                            "calibration requests, averaged over the whole stream",
           "size_scale": args.serving_scale,
           "served": served, "plain": plain, "plain_reused_context": reused,
           "p99_speedup": ratio(plain["p99_latency_s"], served["p99_latency_s"]),
           "shots_per_hour_ratio": ratio(served["shots_per_hour"], plain["shots_per_hour"]),
           "vs_reused_context": {"p99_speedup": ratio(reused["p99_latency_s"], served["p99_latency_s"]),
                                 "shots_per_hour_ratio": ratio(served["shots_per_hour"], reused["shots_per_hour"])}}
    if args.serving_capacity:
        # capacity: the whole stream queued at t = 0
        burst = np.zeros(len(base))
        plain_sat = S.serve_sequential_plain(fresh(), burst)
        served_sat = S.serve_stream(fresh(), burst, slots=args.serving_slots)
        out["capacity"] = {"served_shots_per_hour": served_sat["shots_per_hour"],
                           "plain_shots_per_hour": plain_sat["shots_per_hour"],
                           "served_p99_s": served_sat["p99_latency_s"], "plain_p99_s": plain_sat["p99_latency_s"],
                           "served_errors": served_sat["errors"], "plain_errors": plain_sat["errors"],
                           "ratio": ratio(served_sat["shots_per_hour"], plain_sat["shots_per_hour"])}
    return out


def gradient_alg_bytes(npts, ndamp, nt, nseg):
    """Compulsory HBM bytes of the snapshot gradient (forward with snapshot pairs,
    recompute between them, adjoint with the fused correlation): per time step the
    forward and the recomputed stencil each move 16 B/pt (u^n, u^{n-1}, b read,
    u^{n+1} written) + 4 B/pt where damped (s), the adjoint+gradient stencil the same
    plus 4 B/pt (u^j) and 8 B/pt (gradient read and written); each snapshot pair
    writes 8 B/pt; the gradient is zeroed and copied out once (12 B/pt)."""
    stencil = 16 * npts + 4 * ndamp
    return nt * (2 * stencil + stencil + 12 * npts) + nseg * 8 * npts + 12 * npts


def full_history_alg_bytes(npts, ndamp, nt):
    """The same for the whole-history gradient: the forward stencil's output is the
    stored level (no snapshot copies, no recompute)."""
    stencil = 16 * npts + 4 * ndamp
    return nt * (stencil + stencil + 12 * npts) + 12 * npts


def gradient_leg(args):
    """FWI objective + gradient of one shot on the 3D gradient workload: 200^3
    interior + 40-point layer (280^3), layered model with Gaussian blobs, start
    model smoothed by a 20-point Gaussian, SO8, 1500 steps, snapshots every 10,
    200 x 200 receivers (wp_fwi_gradient_dev, inputs resident in HBM)."""
    import torch
    from paper_1808_01995_gb300 import synth
    from paper_1808_01995_gb300 import wavprop as W
    true, start = synth.blobs_3d()
    k, nt, S = 8, args.gradient_nt, 10
    dt = 0.9 * W.wp_cfl_dt(W.Grid(true.shape, true.spacing, true.origin, k), max(true.vmax, start.vmax))
    grid = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    ctx = W.Context(0)
    q = torch.from_numpy(true.wavelet(dt, nt)).cuda()
    eta = torch.from_numpy(true.eta32()).cuda()
    m_true = torch.from_numpy(true.m32()).cuda()
    d_obs = torch.zeros((nt, len(true.rec)), device="cuda")
    W.wp_forward_dev(ctx.handle, grid, m_true, eta, q, true.src, true.rec, d_obs)
    m0 = torch.from_numpy(start.m32()).cuda()
    g = torch.empty_like(m0)
    J = W.wp_fwi_gradient_dev(ctx.handle, grid, m0, eta, q, true.src, d_obs, true.rec, S, g)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.gradient):
        J = W.wp_fwi_gradient_dev(ctx.handle, grid, m0, eta, q, true.src, d_obs, true.rec, S, g)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.gradient
    npts = int(np.prod(true.shape))
    ndamp = int(np.count_nonzero(true.eta))
    nseg = -(-nt // S)
    peak = W.wp_bytes_in_use(ctx.handle)
    # the same gradient with binomial checkpointing (given residual, own context for its memory)
    d0 = torch.zeros_like(d_obs)
    W.wp_forward_dev(ctx.handle, grid, m0, eta, q, true.src, true.rec, d0)
    r = (d0 - d_obs).contiguous()
    ctx.close()
    ck = {}
    if args.checkpoints > 0:
        cctx = W.Context(0)
        gc = torch.empty_like(m0)
        W.wp_gradient_checkpointed_dev(cctx.handle, grid, m0, eta, q, true.src, r, true.rec, args.checkpoints, gc)
        torch.cuda.synchronize()
        e0.record()
        W.wp_gradient_checkpointed_dev(cctx.handle, grid, m0, eta, q, true.src, r, true.rec, args.checkpoints, gc)
        e1.record()
        torch.cuda.synchronize()
        _, fw = W.wp_checkpoint_schedule(nt, args.checkpoints)
        ck = {"checkpoints": args.checkpoints, "ms_per_gradient": e0.elapsed_time(e1),
              "device_bytes": int(W.wp_bytes_in_use(cctx.handle)), "forward_steps": fw,
              "same_as_snapshots": bool(torch.equal(gc, g))}
        cctx.close()
    fh = {}
    if args.full_history:
        hctx = W.Context(0)
        gh = torch.empty_like(m0)
        W.wp_fwi_gradient_dev(hctx.handle, grid, m0, eta, q, true.src, d_obs, true.rec, 1, gh)
        torch.cuda.synchronize()
        e0.record()
        W.wp_fwi_gradient_dev(hctx.handle, grid, m0, eta, q, true.src, d_obs, true.rec, 1, gh)
        e1.record()
        torch.cuda.synchronize()
        fh = {"ms_per_gradient": e0.elapsed_time(e1), "device_bytes": int(W.wp_bytes_in_use(hctx.handle)),
              "same_as_snapshots": bool(torch.equal(gh, g)),
              "passes": "forward writing every level once + adjoint with fused correlation (no recompute)"}
        hctx.close()
    rc = {}
    if args.reconstruct:
        rctx = W.Context(0)
        gr = torch.empty_like(m0)
        W.wp_gradient_reconstruct_dev(rctx.handle, grid, m0, eta, q, true.src, r, true.rec, gr)
        torch.cuda.synchronize()
        e0.record()
        W.wp_gradient_reconstruct_dev(rctx.handle, grid, m0, eta, q, true.src, r, true.rec, gr)
        e1.record()
        torch.cuda.synchronize()
        nb = true.nbl
        inner = (slice(nb, -nb),) * 3
        a, b = gr[inner].double(), g[inner].double()
        rc = {"ms_per_gradient": e0.elapsed_time(e1), "device_bytes": int(W.wp_bytes_in_use(rctx.handle)),
              "rel_l2_vs_snapshots_interior": float((a - b).norm() / b.norm())}
        rctx.close()
    hbm, hbm_kind = measured_peaks()
    alg = gradient_alg_bytes(npts, ndamp, nt, nseg)
    roof = {"bound": "hbm", "alg_bytes": alg, "bytes_per_point_step": alg / (npts * nt),
            "achieved": alg / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": alg / (ms * 1e-3) / 1e9 / hbm, "peak_source": hbm_kind,
            "counted": "per step: forward stencil 16 B/pt + 4 B/pt damped, recompute the same, adjoint stencil "
                       "the same + u^j read 4 B/pt + gradient read-modify-write 8 B/pt; 8 B/pt per snapshot pair; "
                       "12 B/pt once (gradient zeroed, copied out)"}
    if fh:
        alg_fh = full_history_alg_bytes(npts, ndamp, nt)
        fh["roofline"] = {"alg_bytes": alg_fh, "achieved": alg_fh / (fh["ms_per_gradient"] * 1e-3) / 1e9,
                          "frac": alg_fh / (fh["ms_per_gradient"] * 1e-3) / 1e9 / hbm, "peak": hbm,
                          "counted": "forward stencil (its output is the stored level) + adjoint stencil with "
                                     "u^j read and gradient read-modify-write, per step"}
    return {"workload": f"blobs3d 200^3 + 40 ({true.shape[0]}^3) SO8, nt={nt}, snapshots every {S}, "
                        f"{len(true.rec)} receivers", "ms_per_gradient": ms,
            "gpts_per_s": npts * nt / (ms * 1e-3) / 1e9, "misfit": J, "device_bytes": int(peak),
            "passes": "forward with snapshots + recompute + adjoint with fused correlation",
            "roofline": roof,
            "full_history": fh, "binomial_checkpointing": ck, "boundary_reconstruction": rc}


def large_leg(args):
    """The SO16 salt workload at full size: 512 x 512 x 400 interior + 40-point layer
    (592 x 592 x 480, 168 M points), 3000 steps, 256 x 256 receivers: one forward
    shot and one FWI gradient with snapshots every 20 steps (about 220 GB)."""
    import torch
    from paper_1808_01995_gb300 import synth
    from paper_1808_01995_gb300 import wavprop as W
    torch.cuda.empty_cache()
    true = synth.salt_3d()
    k, nt, S = 16, args.large_nt, 20
    dt = 0.9 * W.wp_cfl_dt(W.Grid(true.shape, true.spacing, true.origin, k), true.vmax)
    grid = W.Grid(true.shape, true.spacing, true.origin, k, dt, nt)
    need = W.wp_estimate_bytes(grid, 1, len(true.rec), 1, S)
    free, _ = torch.cuda.mem_get_info()
    desc = f"salt3d 512x512x400 + 40 ({'x'.join(map(str, true.shape))}) SO16, nt={nt}, {len(true.rec)} receivers"
    if need > 0.85 * free:
        return {"workload": desc, "skipped": f"needs {need / 2**30:.0f} GiB, {free / 2**30:.0f} GiB free"}
    ctx = W.Context(0)
    m = torch.from_numpy(true.m32()).cuda()
    eta = torch.from_numpy(true.eta32()).cuda()
    q = torch.from_numpy(true.wavelet(dt, nt)).cuda()
    d = torch.zeros((nt, len(true.rec)), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    W.wp_forward_dev(ctx.handle, grid, m, eta, q, true.src, true.rec, d)
    torch.cuda.synchronize()
    e0.record()
    W.wp_forward_dev(ctx.handle, grid, m, eta, q, true.src, true.rec, d)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    g = torch.empty_like(m)
    d_obs = torch.zeros_like(d)
    W.wp_fwi_gradient_dev(ctx.handle, grid, m, eta, q, true.src, d_obs, true.rec, S, g)
    torch.cuda.synchronize()
    e0.record()
    J = W.wp_fwi_gradient_dev(ctx.handle, grid, m, eta, q, true.src, d_obs, true.rec, S, g)
    e1.record()
    torch.cuda.synchronize()
    grad_ms = e0.elapsed_time(e1)
    npts = int(np.prod(true.shape))
    out = {"workload": desc, "forward_ms": fwd_ms, "forward_gpts_per_s": npts * nt / (fwd_ms * 1e-3) / 1e9,
           "gradient_ms": grad_ms, "gradient_snap_interval": S, "misfit": J,
           "device_bytes": int(W.wp_bytes_in_use(ctx.handle))}
    ctx.close()
    del m, eta, q, d, g, d_obs
    torch.cuda.empty_cache()
    return out


# The paper's time-to-solution experiment (Sec. 6.2): 1000 ms of modelling at space
# order 16 on an Intel Skylake 8180 (28 cores, 2.5 GHz, STREAM TRIAD 105 GB/s).  The
# paper states neither the velocity model nor dt, so the step counts may differ:
# context, not a baseline.
PAPER_TIME_TO_SOLUTION_S = {512: 17.1, 1024: 162.6}


def paper_context_leg(args):
    """Time to solution of 1000 ms of modelling at SO16 on n^3 grids (n = 512 by
    default; the 40-point damping layer included in n), the layered model of the
    stencil sweep, dt = 0.9 x CFL, one forward shot (coefficients, stencil,
    injection, 128 x 128 receivers), inputs resident in HBM, timed after one
    warm-up shot."""
    import torch
    from paper_1808_01995_gb300 import synth
    from paper_1808_01995_gb300 import wavprop as W
    out = []
    for n in args.context:
        torch.cuda.empty_cache()
        k, nbl = 16, 40
        model = synth.layers_3d(space_order=k, n=n - 2 * nbl, nbl=nbl)
        dt_max = W.wp_cfl_dt(W.Grid(model.shape, model.spacing, model.origin, k), model.vmax)
        nt = int(math.ceil(1.0 / (0.9 * dt_max)))
        dt = 1.0 / nt
        grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
        ctx = W.Context(0)
        m = torch.from_numpy(model.m32()).cuda()
        eta = torch.from_numpy(model.eta32()).cuda()
        q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
        d = torch.zeros((nt, len(model.rec)), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        W.wp_forward_dev(ctx.handle, grid, m, eta, q, model.src, model.rec, d)
        torch.cuda.synchronize()
        e0.record()
        W.wp_forward_dev(ctx.handle, grid, m, eta, q, model.src, model.rec, d)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) * 1e-3
        npts = int(np.prod(model.shape))
        out.append({"grid": list(model.shape), "space_order": k, "modelled_s": 1.0, "nt": nt, "dt_s": dt,
                    "time_to_solution_s": s, "gpts_per_s": npts * nt / s / 1e9,
                    "paper_time_to_solution_s": PAPER_TIME_TO_SOLUTION_S.get(n),
                    "paper_hardware": "Intel Skylake 8180, 28 cores, 2.5 GHz (CPU; dt and model not stated)"})
        ctx.close()
        del m, eta, q, d
        torch.cuda.empty_cache()
    return out


def order_sweep_leg(args, headline):
    """The stencil sweep workload (256^3 + 40-point layer, 1000 steps) at each space
    order of --orders: the shot's rate and the stencil kernel's compulsory bytes
    over its CUDA-event average (every launch bracketed), against the measured HBM
    copy bandwidth.  The headline order reuses the headline run."""
    import torch
    from paper_1808_01995_gb300 import wavprop as W
    peak, peak_kind = measured_peaks()
    out = {}
    for k in args.orders:
        if k == args.space_order and headline is not None:
            out[f"so{k}"] = headline
            continue
        args_k = argparse.Namespace(**vars(args))
        args_k.space_order = k
        model = workload(args_k)
        dt = 0.9 * W.wp_cfl_dt(W.Grid(model.shape, model.spacing, model.origin, k), model.vmax)
        nt = args.nt
        grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
        with W.Context(0) as ctx:
            m = torch.from_numpy(model.m32()).cuda()
            eta = torch.from_numpy(model.eta32()).cuda()
            q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
            rec = torch.zeros((nt, len(model.rec)), device="cuda")
            W.wp_forward_dev(ctx.handle, grid, m, eta, q, model.src, model.rec, rec)
            torch.cuda.synchronize()
            W.wp_set_profiling(ctx.handle, 1)
            W.wp_profile_read(ctx.handle, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.order_shots):
                W.wp_forward_dev(ctx.handle, grid, m, eta, q, model.src, model.rec, rec)
            e1.record()
            torch.cuda.synchronize()
            k_ms, k_n = W.wp_profile_read(ctx.handle, reset=True)
            ms = e0.elapsed_time(e1) / args.order_shots
        alg, npts, _ = algorithmic_bytes_per_launch(model)
        avg_s = k_ms / max(k_n, 1) * 1e-3
        out[f"so{k}"] = {"value": npts * nt / (ms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_shot": ms,
                         "kernel": f"{'stencil3d_kernel' if k <= 8 else 'stencil3d_hi_kernel'}<R={k // 2},fwd>",
                         "kernel_avg_us": avg_s * 1e6, "alg_bytes_per_launch": alg,
                         "achieved": alg / avg_s / 1e9, "peak": peak, "unit_roofline": "GB/s",
                         "frac": alg / avg_s / 1e9 / peak, "peak_source": peak_kind,
                         "traffic": kernel_traffic(k, "x".join(str(s) for s in model.shape)),
                         "timed_launches": k_n}
        del m, eta, q, rec
        torch.cuda.empty_cache()
    return out


def cfd_leg(args):
    """The CFD examples of Sec. 5 at GPU scale: 8192^2 fields (67 M points, 256 MB
    each, larger than L2), convection and Poisson 200 steps, Burgers' equation 100,
    inputs resident in HBM (device-array calls)."""
    import torch
    from paper_1808_01995_gb300 import wavprop as W
    n = args.cfd_n
    rng = np.random.default_rng(1808 + 7)
    dx = dy = 1.0 / (n - 1)
    u0 = torch.from_numpy(rng.uniform(1.0, 2.0, (n, n)).astype(np.float32)).cuda()
    v0 = torch.from_numpy(rng.uniform(0.5, 1.5, (n, n)).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal((n, n)).astype(np.float32)).cuda()
    o1, o2 = torch.empty_like(u0), torch.empty_like(u0)
    ctx = W.Context(0)
    h = ctx.handle
    c, nu = 1.0, 1e-7
    dt = 0.45 / (c / dx + c / dy)
    dtb = 0.4 / (2.0 / dx + 2.0 / dy + 2 * nu * (1 / dx**2 + 1 / dy**2))
    runs = {
        "convection": (200, 8, lambda k: W.wp_convection_2d_dev(h, u0, dx, dy, dt, c, k, o1)),
        "burgers": (100, 16, lambda k: W.wp_burgers_2d_dev(h, u0, v0, dx, dy, dtb, nu, k, o1, o2)),
        "poisson": (200, 12, lambda k: W.wp_poisson_2d_dev(h, u0, b, dx, dy, k, o1)),
    }
    peak, _ = measured_peaks()
    out = {"grid": [n, n], "inputs": "resident in HBM"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, (steps, bpp, fn) in runs.items():
        fn(4)  # warm-up (pool, first launches)
        torch.cuda.synchronize()
        e0.record()
        fn(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        pts = float(n) * n * steps
        gbs = bpp * pts / (ms * 1e-3) / 1e9
        out[name] = {"steps": steps, "ms": ms, "gpts_per_s": pts / (ms * 1e-3) / 1e9,
                     "bytes_per_point_step": bpp, "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak}
    ctx.close()
    return out


def run_ours(args):
    world, rank, local = dist_init()
    import torch
    torch.cuda.set_device(local)
    from paper_1808_01995_gb300 import build as B
    from paper_1808_01995_gb300 import wavprop as W
    if rank == 0:  # one rank builds; the others load the library after the barrier
        B.build()
    barrier(world)
    model = workload(args)
    k = args.space_order
    grid0 = W.Grid(model.shape, model.spacing, model.origin, k)
    dt = 0.9 * W.wp_cfl_dt(grid0, model.vmax)
    nt = args.nt
    grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    ctx = W.Context(local)
    h = ctx.handle
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
    rec = torch.zeros((nt, len(model.rec)), device="cuda")
    src_c, rec_c = model.src, model.rec

    def step():
        W.wp_forward_dev(h, grid, m, eta, q, src_c, rec_c, rec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    W.wp_set_profiling(h, args.profile_every)
    W.wp_profile_read(h, reset=True)
    launches0 = W.wp_kernel_launches(h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    barrier(world)
    launches = W.wp_kernel_launches(h) - launches0
    k_ms, k_n = W.wp_profile_read(h, reset=True)
    W.wp_set_profiling(h, 0)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world)
    npts = int(np.prod(model.shape))
    value = whole_job_rate(world, npts * nt * args.steps, ms * 1e-3)
    nint = int(np.prod([n - 2 * model.nbl for n in model.shape]))
    interior = {"value": value * nint / npts, "unit": "Gpts/s", "points": nint,
                "note": "the same run counted over the physical interior only (damping layer excluded)"}

    alg_bytes, _, ndamp = algorithmic_bytes_per_launch(model)
    peak, peak_kind = measured_peaks()
    k_avg_s = (k_ms / max(k_n, 1)) * 1e-3
    achieved = alg_bytes / k_avg_s / 1e9
    traffic = kernel_traffic(k, "x".join(str(s) for s in model.shape))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": f"{'stencil3d_kernel' if k <= 8 else 'stencil3d_hi_kernel'}<R={k // 2},fwd>",
                "kernel_avg_us": k_avg_s * 1e6, "alg_bytes_per_launch": alg_bytes,
                "timed_launches": k_n, "sampled_every": args.profile_every,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"}

    e2e = None
    if not args.no_e2e:
        mh = torch.from_numpy(model.m32()).pin_memory()
        eh = torch.from_numpy(model.eta32()).pin_memory()
        qh = torch.from_numpy(model.wavelet(dt, nt)).pin_memory()
        mhn, ehn, qhn = mh.numpy(), eh.numpy(), qh.numpy()
        out_h = torch.empty((nt, len(model.rec)), dtype=torch.float32).pin_memory().numpy()
        lib = W.lib()
        import ctypes
        g = grid.c()
        src_a = np.ascontiguousarray(src_c, dtype=np.float64)
        rec_a = np.ascontiguousarray(rec_c, dtype=np.float64)

        def e2e_step():
            rc = lib.wp_forward(h, ctypes.byref(g), mhn.ctypes.data, ehn.ctypes.data, qhn.ctypes.data, len(src_a),
                                src_a.ctypes.data, len(rec_a), rec_a.ctypes.data, out_h.ctypes.data)
            if rc != 0:
                raise RuntimeError(W.wp_last_error())

        e2e_step()
        torch.cuda.synchronize()
        ke = max(1, args.steps)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": whole_job_rate(world, npts * nt * ke, el), "unit": "Gpts/s",
               "h2d_bytes_per_step": int(mhn.nbytes + ehn.nbytes + qhn.nbytes),
               "d2h_bytes_per_step": int(out_h.nbytes), "steps": ke,
               "call": "wp_forward (host arrays, pinned)"}

    # single-GPU legs: reported by the N = 1 run (replicas add nothing to them)
    by_order = None
    if args.orders and world == 1:
        head = {"value": value, "unit": "Gpts/s", "ms_per_shot": ms / args.steps, "kernel": roofline["kernel"],
                "kernel_avg_us": roofline["kernel_avg_us"], "alg_bytes_per_launch": alg_bytes,
                "achieved": achieved, "peak": peak, "unit_roofline": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "traffic": traffic, "timed_launches": k_n,
                "note": "the headline run (launches sampled every --profile-every)"}
        by_order = order_sweep_leg(args, head)

    gradient = None
    if args.gradient > 0 and world == 1:
        gradient = gradient_leg(args)

    serving = None
    if args.serving > 0 and world == 1:
        serving = serving_leg(args)

    large = None
    if args.large_nt > 0 and world == 1:
        large = large_leg(args)

    cfd = None
    if args.cfd_n > 0 and world == 1:
        cfd = cfd_leg(args)

    context = None
    if args.context and world == 1:
        context = paper_context_leg(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, steps, el, nthreads = oracle_sample(model, dt, args.cpu_seconds)
        cpu = {"value": rate, "unit": "Gpts/s", "cores": nthreads, "kind": "oracle",
               "sample": f"FP64 oracle forward on the full grid, {steps} of {nt} time steps ({el:.1f} s)"}
        rate1, steps1, el1 = oracle_sample_one_thread(model, dt, nthreads)
        cpu["value_1thread"] = rate1
        cpu["sample_1thread"] = f"the same on one thread, {steps1} time steps ({el1:.1f} s)"

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": describe(model, nt, dt),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "value_interior": interior,
                "clocks": clk.summary(), "roofline_by_order": by_order, "gradient": gradient, "serving": serving, "large": large, "cfd": cfd, "paper_context": context}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
