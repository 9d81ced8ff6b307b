"""Programmatic dependent launch in the time loop.

Inside a time loop the injection, interpolation and the next step's stencil are
launched with programmatic stream serialization: each may start launching while
the kernel before it still runs, and waits on the device for that kernel to
complete before touching memory.  The order of every read and write is the same
as with ordinary launches, so receiver data must be equal bit for bit with it on
(the default) and off (WP_PDL=0, read when a context is created), in replayed
graphs (nt >= 16) and in plain launches (a short loop), at an order of each
stencil kernel, and with the profiling event records that break the chain.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1808_01995_gb300 import synth
from paper_1808_01995_gb300 import wavprop as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_01995_gb300 import build
    build.build()


def context(pdl):
    old = os.environ.get("WP_PDL")
    os.environ["WP_PDL"] = pdl
    try:
        return W.Context(0)
    finally:
        if old is None:
            os.environ.pop("WP_PDL")
        else:
            os.environ["WP_PDL"] = old


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("k,nt,profile", [(8, 70, 0), (8, 9, 0), (16, 40, 0), (8, 70, 3), (4, 36, 0)])
def test_receiver_data_equal_with_and_without_programmatic_launch(k, nt, profile):
    model = synth.random_case((36, 41, 66), k, nsrc=2, nrec=30, nbl=5, seed=50 + k + nt)
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
    outs = []
    for pdl in ("1", "0"):
        c = context(pdl)
        try:
            if profile:
                W.wp_set_profiling(c.handle, profile)
            for _ in range(2):  # the second call replays the cached graphs
                out = torch.full((nt, len(model.rec)), float("nan"), device="cuda")
                W.wp_forward_dev(c.handle, grid, m, eta, q, model.src, model.rec, out)
                torch.cuda.synchronize()
                outs.append(out.cpu().numpy())
        finally:
            c.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    og = O.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    ref = O.forward(og, model.m32(), model.eta32(), model.wavelet(dt, nt), model.src, model.rec)
    assert rel_l2(outs[0], ref) < 1e-4


def test_gradient_equal_with_and_without_programmatic_launch():
    # the forward pass that writes snapshots, the recomputation and the
    # adjoint+gradient steps all run as chains of step kernels
    k, nt = 8, 48
    model = synth.random_case((34, 38, 60), k, nsrc=2, nrec=21, nbl=5, seed=61)
    dt = 0.9 * O.cfl_dt(model.spacing, k, model.vmax)
    grid = W.Grid(model.shape, model.spacing, model.origin, k, dt, nt)
    m = torch.from_numpy(model.m32()).cuda()
    eta = torch.from_numpy(model.eta32()).cuda()
    q = torch.from_numpy(model.wavelet(dt, nt)).cuda()
    res = torch.from_numpy(np.random.default_rng(62).standard_normal((nt, len(model.rec))).astype(np.float32)).cuda()
    grads = []
    for pdl in ("1", "0"):
        c = context(pdl)
        try:
            g = torch.zeros(model.shape, device="cuda")
            W.wp_gradient_dev(c.handle, grid, m, eta, q, model.src, res, model.rec, 6, g)
            torch.cuda.synchronize()
            grads.append(g.cpu().numpy())
        finally:
            c.close()
    assert np.abs(grads[1]).max() > 0
    assert np.array_equal(grads[0], grads[1])
